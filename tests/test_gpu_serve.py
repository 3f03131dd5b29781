"""Serving loop: requests that arrive while others run are admitted by HBM
budget and overlap on the GPU (continuous batching); each result is the same
alone and in the mix, and matches the FP64 oracle (runs of up to 18 qubits);
budget rejection and cancellation work."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1910_08020_gb300 as z2
from oracle.lattice import Lattice as OLattice
from paper_1910_08020_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    z2.build()
    c = z2.Context(0)
    yield c.handle
    c.close()


def fields(r):
    return np.array([r.energy, r.norm, r.mean_plaq, r.mean_star] + list(r.plaq[:12]) + list(r.sigmax[:24]))


def stream(count, seed):
    reqs = workloads.poisson_stream(count, rate=400.0, seed=seed,
                                    lattices=[(2, (2, 2)), (2, (3, 2)), (2, (4, 2)), (2, (3, 3)), (2, (4, 3))],
                                    m_range=(10, 60))
    return reqs


def test_serve_mix_equals_alone(ctx):
    reqs = stream(24, 3)
    # answers alone first (plain runs through the same context)
    alone = []
    for rq in reqs:
        lat = z2.Lattice(rq["d"], rq["L"])
        g = torch.empty(1 << lat.n_links, dtype=torch.complex64, device="cuda")
        alone.append(fields(z2.z2_run(ctx, lat.handle, z2.params(rq["lam"], rq["T"], rq["M"]), g)))
        del g
    torch.cuda.synchronize()
    srv = z2.z2_server_create(ctx, hbm_budget=512 << 20, max_slots=4)
    try:
        t0 = time.monotonic()
        tickets = []
        for rq in reqs:  # arrivals on the request stream's clock
            delay = rq["arrival"] - (time.monotonic() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(z2.z2_server_submit(srv, rq))
        for tk, want in zip(tickets, alone):
            rc, res = z2.z2_server_wait(srv, tk, timeout_s=120)
            assert rc == 0
            assert np.array_equal(fields(res), want)
            q, r = z2.z2_server_request_times(srv, tk)
            assert q >= 0 and r > 0
        st = z2.z2_server_stats(srv)
        assert st.submitted == st.completed == len(reqs)
        assert st.hbm_peak <= 512 << 20 and st.hbm_in_use == 0 and st.active == 0
        # each served result against the FP64 oracle (lattices of <= 18 links),
        # at the run tolerances: 1e-5 (bounded observables), 1e-5 (N + lambda N_p)
        # for the energy
        checked = 0
        for tk, rq in zip(tickets, reqs):
            ol = OLattice(rq["d"], rq["L"])
            if ol.n_links > 18:
                continue
            _, res = z2.z2_server_wait(srv, tk, timeout_s=10)
            d = z2.results_dict(res, z2.Lattice(rq["d"], rq["L"]).info)
            ref = oracle.observables(ol, oracle.run(ol, rq["lam"], rq["T"], rq["M"], 1), rq["lam"])
            S = ol.n_links + abs(rq["lam"]) * ol.n_plaq
            assert abs(d["energy"] - ref["energy"]) < 1e-5 * S
            assert abs(d["norm"] - ref["norm"]) < 1e-5
            assert np.max(np.abs(d["plaq"] - ref["plaq"])) < 1e-5
            assert np.max(np.abs(d["sigmax"] - ref["sigmax"])) < 1e-5
            assert np.max(np.abs(d["star"] - ref["star"])) < 1e-5
            checked += 1
        assert checked >= 10
    finally:
        z2.z2_server_destroy(srv)


def test_served_runs_overlap_on_device(ctx):
    # Two 24-qubit runs submitted together to a two-slot server: the second
    # run's first kernel completes while the first run is still on the GPU
    # (device-clock events on the runs' streams), which a server that ran one
    # request at a time could not show.
    srv = z2.z2_server_create(ctx, hbm_budget=1 << 30, max_slots=2)
    try:
        spec = dict(d=2, L=(4, 3), lam=2.0, T=8.0, M=200)
        tks = [z2.z2_server_submit(srv, spec) for _ in range(2)]
        iv = []
        for tk in tks:
            rc, res = z2.z2_server_wait(srv, tk, timeout_s=120)
            assert rc == 0 and abs(res.norm - 1) < 1e-5
            iv.append(z2.z2_server_request_device_times(srv, tk))
        (a0, a1), (b0, b1) = iv
        assert a0 < a1 and b0 < b1
        both = min(a1, b1) - max(a0, b0)
        assert both > 0.25 * min(a1 - a0, b1 - b0), iv
    finally:
        z2.z2_server_destroy(srv)


def test_serve_budget_and_cancel(ctx):
    srv = z2.z2_server_create(ctx, hbm_budget=64 << 20, max_slots=1)
    try:
        big = dict(d=2, L=(4, 3), lam=1.0, T=1.0, M=10)  # 128 MB state > budget
        with pytest.raises(z2.Z2Error) as e:
            z2.z2_server_submit(srv, big)
        assert e.value.code == -4
        small = dict(d=2, L=(3, 3), lam=1.0, T=4.0, M=400)
        tks = [z2.z2_server_submit(srv, small) for _ in range(6)]
        assert z2.z2_server_cancel(srv, tks[-1]) == 0
        rc, _ = z2.z2_server_wait(srv, tks[-1], timeout_s=60)
        assert rc == -7
        for tk in tks[:-1]:
            rc, res = z2.z2_server_wait(srv, tk, timeout_s=120)
            assert rc == 0 and abs(res.norm - 1) < 1e-5
        st = z2.z2_server_stats(srv)
        assert st.rejected == 1 and st.cancelled == 1 and st.completed == 5
    finally:
        z2.z2_server_destroy(srv)


def test_size_classes_large_runs_take_turns(ctx):
    # With one large-run place, two 24-qubit runs never share the GPU: the
    # second one's first kernel runs after the first one's work has ended.
    # A small run submitted after both passes the waiting one and runs beside
    # the first (device-clock events on the runs' streams).
    srv = z2.z2_server_create(ctx, hbm_budget=1 << 30, max_slots=4)
    try:
        z2.z2_server_set_option(srv, z2.Z2_SERVE_OPT_MAX_LARGE, 1)
        big = dict(d=2, L=(4, 3), lam=2.0, T=8.0, M=200)
        small = dict(d=2, L=(3, 3), lam=1.0, T=2.0, M=50)
        tbig = [z2.z2_server_submit(srv, big) for _ in range(2)]
        tsmall = z2.z2_server_submit(srv, small)
        for tk in tbig + [tsmall]:
            rc, res = z2.z2_server_wait(srv, tk, timeout_s=120)
            assert rc == 0 and abs(res.norm - 1) < 1e-5
        (a0, a1), (b0, b1) = (z2.z2_server_request_device_times(srv, tk) for tk in tbig)
        s0, s1 = z2.z2_server_request_device_times(srv, tsmall)
        assert b0 > a1, ((a0, a1), (b0, b1))
        assert s0 < a1, ((a0, a1), (s0, s1))
        with pytest.raises(z2.Z2Error):
            z2.z2_server_set_option(srv, z2.Z2_SERVE_OPT_MAX_LARGE, 0)
        with pytest.raises(z2.Z2Error):
            z2.z2_server_set_option(srv, 7, 1)
    finally:
        z2.z2_server_destroy(srv)
