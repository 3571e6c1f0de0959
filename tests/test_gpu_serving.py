"""Several problems on one GPU: fine sweeps of several contexts in one persistent launch
(pr_fine_sweep_batch), the fine-launch autotuner (pr_tune_fine) and the continuous-
batching server (pr_server_*).  Each result must be the same alone and in the mix; with a
fixed CTA-group size the kernels take identical steps, so the results are bit-identical.
"""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from test_gpu_parity import rel

pytestmark = pytest.mark.gpu


def mix():
    """Two problems on a 16^3 grid (different flow, eps, horizon, subintervals, forcing)
    and one on an 8^3 grid."""
    a = pi.tiny(n=16, n_sub=6, flow=pi.Flow("abc"), eps=0.05, T=0.12, name="a")
    b = pi.tiny(n=16, n_sub=4, flow=pi.Flow("kolmogorov", k=2), eps=0.02, T=0.08, f_seed=3,
                name="b")
    c = pi.tiny(n=8, n_sub=4, name="c")
    return a, b, c


def started(bd, w, prec, **kw):
    s = bd.Parareal.from_workload(w, precision=prec, **kw)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    return s


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_batched_fine_sweep_equals_single_sweeps(gpu, prec):
    bd, torch = gpu
    a, b, _ = mix()
    single = {}
    for w in (a, b):
        s = started(bd, w, prec, group_ctas=4)
        s.fine_sweep(1)
        single[w.name] = ([s.fine_end(n) for n in range(w.n_sub)],
                          [s.snapshots(n) for n in range(w.n_sub)])
        s.close()
    sa, sb = started(bd, a, prec, group_ctas=4), started(bd, b, prec, group_ctas=4)
    bd.fine_sweep_batch([sa, sb], [1, 1])
    for s, w in ((sa, a), (sb, b)):
        F, W = single[w.name]
        for n in range(w.n_sub):
            assert np.array_equal(s.fine_end(n), F[n]), (w.name, n)
            assert np.array_equal(s.snapshots(n), W[n]), (w.name, n)
    # both iterations carry on from the batched sweep
    for s in (sa, sb):
        s.pod_update(1)
        s.coarse_sweep(1)
        s.check(1)
    sa.close()
    sb.close()


def test_batched_fine_sweep_rejects_mixed_shapes_and_order(gpu):
    bd, torch = gpu
    a, _, c = mix()
    sa, sc = started(bd, a, 0), started(bd, c, 0)
    with pytest.raises(bd.PRError):
        bd.fine_sweep_batch([sa, sc], [1, 1])        # different n
    with pytest.raises(bd.PRError):
        bd.fine_sweep_batch([sa, sa], [1, 1])        # the same context twice
    with pytest.raises(bd.PRError):
        bd.fine_sweep_batch([sa], [2])               # out of order
    sa.close()
    sc.close()


def test_tune_fine_keeps_the_iterate_and_fixes_the_group_size(gpu):
    bd, torch = gpu
    w = pi.tiny(n=16, n_sub=4)
    s = started(bd, w, 0)
    U0 = s.interfaces()
    G, ms = s.tune_fine(4)
    assert G >= 1 and ms > 0
    assert np.array_equal(s.interfaces(), U0)
    s.iterate(1)
    r = started(bd, w, 0, group_ctas=G)
    r.iterate(1)
    assert np.array_equal(s.interfaces(), r.interfaces())
    s.close()
    r.close()


def run_server(bd, reqs, prec, tol, **srv_kw):
    import time
    srv = bd.Server(**srv_kw)
    ids = [srv.submit(w, w.u0(), w.f(), tol=tol, precision=prec, group_ctas=4) for w in reqs]
    most_active = 0
    t0 = time.time()
    while True:
        act, pend = srv.step()
        most_active = max(most_active, act)
        if act == 0 and pend == 0:
            break
        assert time.time() - t0 < 120
    out = {}
    for w, i in zip(reqs, ids):
        st, k, inc = srv.query(i)
        assert st == bd.PR_REQ_DONE, srv.request_error(i)
        out[w.name] = (srv.result(i), k, inc)
    srv.close()
    return out, most_active


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_server_result_is_the_same_alone_and_in_the_mix(gpu, prec):
    bd, torch = gpu
    reqs = mix()
    tol = 1e-9 if prec == 0 else 1e-6
    together, most = run_server(bd, reqs, prec, tol)
    assert most == 3
    for w in reqs:
        alone, _ = run_server(bd, [w], prec, tol)
        assert np.array_equal(together[w.name][0], alone[w.name][0]), w.name
        assert together[w.name][1] == alone[w.name][1]
    # one at a time (resident cap 1): same results, requests wait for a slot
    serial, most = run_server(bd, reqs, prec, tol, max_active=1)
    assert most == 1
    for w in reqs:
        assert np.array_equal(serial[w.name][0], together[w.name][0])


def test_server_matches_direct_iterations_and_the_oracle(gpu):
    bd, torch = gpu
    reqs = mix()
    tol = 1e-9
    out, _ = run_server(bd, reqs, 0, tol)
    for w in reqs:
        res, k, inc = out[w.name]
        assert inc <= tol or k == w.n_sub
        s = started(bd, w, 0, group_ctas=4)
        for kk in range(1, k + 1):
            s.iterate(kk)
        assert np.array_equal(s.interface(w.n_sub), res)
        s.close()
    # the oracle's iterate k at the end of the horizon, FP64 mode
    w = reqs[2]
    res, k, _ = out[w.name]
    prm = O.derive_params(w)
    h = O.parareal(w, prm, k_max=k)
    assert rel(res, h["U"][k][w.n_sub]) < 1e-10


def test_server_admission_and_failures(gpu):
    bd, torch = gpu
    a, b, c = mix()
    srv = bd.Server(hbm_budget=1)
    i = srv.submit(c, c.u0(), c.f(), tol=1e-6)
    srv.step()
    st, _, _ = srv.query(i)
    assert st == bd.PR_REQ_FAILED and "budget" in srv.request_error(i)
    with pytest.raises(bd.PRError):
        srv.result(i)
    srv.close()
    # an invalid request fails on its own, the others finish
    bad = pi.tiny(n=8, n_sub=4, T=-1.0, name="bad")
    srv = bd.Server()
    ib = srv.submit(bad, bad.u0(), None, tol=1e-6)
    ic = srv.submit(c, c.u0(), c.f(), tol=1e-6)
    import time
    t0 = time.time()
    while time.time() - t0 < 60:
        act, pend = srv.step()
        if act == 0 and pend == 0:
            break
    assert srv.query(ib)[0] == bd.PR_REQ_FAILED
    assert srv.query(ic)[0] == bd.PR_REQ_DONE
    srv.close()


def test_small_request_finishes_while_a_large_one_is_mid_solve(gpu):
    """Requests run on their own iteration clocks: a small problem submitted beside a
    large one does many iterations while the large one does few, finishes first, and the
    large one's result is still the one it gives alone."""
    import time
    bd, torch = gpu
    big = pi.Workload("big", 48, pi.Flow("abc"), 0.01, 2.0, 32, 1e-3, n_snap=16, m_cap=8)
    small = pi.tiny(n=8, n_sub=4, name="small")
    srv = bd.Server()
    ib = srv.submit(big, big.u0(), None, tol=1e-13, precision=0, group_ctas=4)
    is_ = srv.submit(small, small.u0(), None, tol=1e-9, precision=0, group_ctas=4)
    t0 = time.time()
    while srv.query(is_)[0] not in (bd.PR_REQ_DONE, bd.PR_REQ_FAILED):
        srv.step()
        assert time.time() - t0 < 60
    st_s, k_s, _ = srv.query(is_)
    st_b, k_b, _ = srv.query(ib)
    assert st_s == bd.PR_REQ_DONE, srv.request_error(is_)
    assert st_b == bd.PR_REQ_ACTIVE and k_b < k_s, (k_b, k_s)   # mid-solve, behind
    while srv.query(ib)[0] == bd.PR_REQ_ACTIVE:
        srv.step()
        assert time.time() - t0 < 120
    assert srv.query(ib)[0] == bd.PR_REQ_DONE, srv.request_error(ib)
    res_b, res_s = srv.result(ib), srv.result(is_)
    srv.close()
    alone, _ = run_server(bd, [small], 0, 1e-9)
    assert np.array_equal(alone["small"][0], res_s)
    srv = bd.Server()
    i = srv.submit(big, big.u0(), None, tol=1e-13, precision=0, group_ctas=4)
    while srv.query(i)[0] == bd.PR_REQ_ACTIVE or srv.query(i)[0] == bd.PR_REQ_PENDING:
        srv.step()
        assert time.time() - t0 < 240
    assert np.array_equal(srv.result(i), res_b)
    srv.close()
