"""Host-side logic (no GPU): the cost model against the paper's printed tables, the
bench's traffic model and clock parsing, and the multi-rank reduction on gloo."""
import os

import pytest

from paper_2601_10981_gb300 import report

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cost_tables.txt")


def rows(kind):
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == kind:
            yield f


@pytest.mark.parametrize("row", list(rows("adap")) + list(rows("plain2")), ids=lambda r: "-".join(r[:3]))
def test_iteration_total_reproduces_paper_tables(row):
    T_F, T_G, T_U, T_C, T_A, T_tot = map(float, row[3:9])
    assert abs(report.iteration_total(T_F, T_G, T_U, T_C, T_A, 200) - T_tot) < 0.006


def test_speedup_estimate_reproduces_paper():
    (row,) = list(rows("speedup"))
    T_F, N, T_tot, k, expect = float(row[3]), int(row[4]), float(row[5]), int(row[6]), float(row[7])
    assert abs(report.speedup_estimate(T_F, N, T_tot, k) - expect) < 0.005


def test_cost_par_closed_form_sum():
    # the per-iteration sum equals the closed form with (N - (k_max+1)/2) of Sec. 3.3
    N, kmax, DT, T0, dt, dT = 200, 9, 5.0, 5.0, 1e-2, 0.5
    tF, tG, TC, TU, TA = 0.08, 0.004, 1.0, 1.3, 0.13
    c = report.cost_par(N, kmax, DT, T0, dt, dT, tF, tG, TC, TU, TA)
    closed = (T0 / dt * tF + TC + TU + N * DT / dT * tG
              + kmax * (DT / dt * tF + TC + TU + (N - (kmax + 1) / 2) * (TA + DT / dT * tG)))
    assert abs(c - closed) < 1e-9 * closed


def test_speedup_model_limits():
    # without the augmentation term the speedup is N / k
    assert report.speedup_model(200, 10, 50, 1e-2, 5.0, 0.0) == 20.0
    assert report.speedup_model(200, 10, 50, 1e-2, 5.0, 1e-3) < 20.0


def test_fine_traffic_model():
    import bench
    # FP32: 16 + 12 + 8 (f) + 17*4*n_it + 4/dM
    assert bench.fine_bytes_per_dof_step(4, 3.0, 5, True) == 16 + 12 + 4 + 204 + 1.6
    assert bench.fine_bytes_per_dof_step(8, 2.0, 4, False) == 16 + 24 + 272 + 2
    # a stored velocity perturbation: three words at the setup's stencil and at two per
    # BiCGStab iteration
    assert bench.fine_bytes_per_dof_step(4, 1.0, 41, False, True) == 16 + 12 + 68 + 8 / 41 + 36


def test_clock_sampler_parses_reasons():
    import bench
    cs = bench.ClockSampler(0)
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=0: 0})()
    cs.lines = ["0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active",
                "0, 1980, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1995, 2070, 990.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = cs.stop()
    assert out["sm_mhz"] == 1980 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max(10.0 + rank, dist, "cpu")
    q.put((rank, t))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: 11.0, 1: 11.0}
