"""Batched lambda sweep (z2_sweep): every mode gives each run exactly the
result it has alone (same kernels on the same data in the same order), and
the results agree with the FP64 oracle."""

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


def small_specs(count=12, seed=5):
    # the sweep's recipe with short schedules (oracle-sized) and small lattices
    specs = workloads.sweep_specs(count, seed=seed,
                                  lattices=[(2, (3, 3)), (2, (3, 2)), (2, (2, 2)), (2, (4, 2))])
    for sp in specs:
        sp["M"] = 10 + sp["M"] % 17
        sp["T"] = 0.1 * sp["M"]
    return specs


def fields(r):
    return np.array([r.energy, r.norm, r.mean_plaq, r.mean_star] + list(r.plaq[:9]) + list(r.sigmax[:18]))


@pytest.mark.parametrize("mode", [z2.Z2_SWEEP_PLAIN, z2.Z2_SWEEP_STREAMS, z2.Z2_SWEEP_GRAPHS])
def test_sweep_equals_single_runs(ctx, mode):
    specs = small_specs()
    res = z2.z2_sweep(ctx, specs, mode=mode, n_streams=4)
    for sp, r in zip(specs, res):
        assert r.status == 0
        lat = z2.Lattice(sp["d"], sp["L"])
        g = torch.empty(1 << lat.n_links, dtype=torch.complex64, device="cuda")
        alone = z2.z2_run(ctx, lat.handle, z2.params(sp["lam"], sp["T"], sp["M"]), g)
        assert np.array_equal(fields(r), fields(alone))


def test_sweep_against_oracle(ctx):
    specs = small_specs(6, seed=9)
    res = z2.z2_sweep(ctx, specs, mode=z2.Z2_SWEEP_GRAPHS, n_streams=3)
    for sp, r in zip(specs, res):
        ol = OLattice(sp["d"], sp["L"])
        ref = oracle.observables(ol, oracle.run(ol, sp["lam"], sp["T"], sp["M"], 1), sp["lam"])
        S = ol.n_links + sp["lam"] * ol.n_plaq
        assert abs(r.energy - ref["energy"]) < 1e-5 * S
        assert np.max(np.abs(np.array(r.plaq[:ol.n_plaq]) - ref["plaq"])) < 1e-5


def test_sweep_paper_mix_invariants(ctx):
    # the 18q / 24q mix of the benchmark sweep, shortened: gauge invariants hold
    specs = workloads.sweep_specs(8)
    for sp in specs:
        sp["M"] = 20
        sp["T"] = 1.0
    res = z2.z2_sweep(ctx, specs, mode=z2.Z2_SWEEP_STREAMS, n_streams=4)
    for sp, r in zip(specs, res):
        n_sites = int(np.prod(sp["L"]))
        assert r.status == 0
        assert abs(r.norm - 1) < 1e-5
        assert np.max(np.abs(np.array(r.star[:n_sites]) - 1)) < 1e-5


def test_sweep_errors(ctx):
    specs = small_specs(2)
    specs[1]["M"] = 0
    with pytest.raises(z2.Z2Error):
        z2.z2_sweep(ctx, specs)
    with pytest.raises(z2.Z2Error):
        z2.z2_sweep(ctx, small_specs(2), mode=7)


def test_persistent_sweep(ctx):
    # runs of 14 to 21 qubits go through the one persistent launch (2^14-amplitude
    # tiles, direct kernel arithmetic), the others through the normal path
    specs = small_specs(16, seed=11)
    res = z2.z2_sweep(ctx, specs, mode=z2.Z2_SWEEP_PERSISTENT, n_streams=4)
    for sp, r in zip(specs, res):
        assert r.status == 0
        lat = z2.Lattice(sp["d"], sp["L"])
        g = torch.empty(1 << lat.n_links, dtype=torch.complex64, device="cuda")
        default = z2.z2_run(ctx, lat.handle, z2.params(sp["lam"], sp["T"], sp["M"]), g)
        # same kernel arithmetic as a single run evolved with the same tiles
        # (observables with the context's default plans, as in the sweep)
        p = z2.params(sp["lam"], sp["T"], sp["M"])
        if lat.n_links >= 14:
            z2.z2_ctx_set_option(ctx, z2.Z2_OPT_TILE_BITS, 14)
            z2.z2_ctx_set_option(ctx, z2.Z2_OPT_PASS_VARIANT, 1)
        z2.z2_init_plus(ctx, lat.handle, z2.Z2_C64, g)
        z2.z2_evolve(ctx, lat.handle, p, g, 0, sp["M"])
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_TILE_BITS, 0)
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_PASS_VARIANT, 0)
        same = z2.z2_measure(ctx, lat.handle, p, g)
        assert np.array_equal(fields(r), fields(same))
        assert np.max(np.abs(fields(r) - fields(default))) < 1e-5 * (lat.n_links + sp["lam"] * lat.n_plaq)


def test_persistent_sweep_paper_mix(ctx):
    # the benchmark's lattices (18 and 24 qubits), shortened schedules, vs the oracle where small
    specs = workloads.sweep_specs(10, seed=4)
    for sp in specs:
        sp["M"] = 8
        sp["T"] = 0.4
    res = z2.z2_sweep(ctx, specs, mode=z2.Z2_SWEEP_PERSISTENT, n_streams=3)
    for sp, r in zip(specs, res):
        assert r.status == 0
        n_sites = int(np.prod(sp["L"]))
        assert abs(r.norm - 1) < 1e-5
        assert np.max(np.abs(np.array(r.star[:n_sites]) - 1)) < 1e-5
        if sp["L"] == (3, 3):
            ol = OLattice(sp["d"], sp["L"])
            ref = oracle.observables(ol, oracle.run(ol, sp["lam"], sp["T"], sp["M"], 1), sp["lam"])
            assert abs(r.energy - ref["energy"]) < 1e-5 * (ol.n_links + sp["lam"] * ol.n_plaq)


def test_persistent_gang_wait_runs_out_then_recovers(ctx):
    # Failure detection without a GPU fault.  The persistent kernel's gang
    # barrier is a bounded poll of a counter in global memory, with no copies
    # in flight.  With the limit at one poll, a CTA that reaches a barrier
    # before the rest of its gang gives up at once, sets the device error
    # flag and returns; the gang's other CTAs give up at their next barrier,
    # and the call reports Z2_ERR_DEVICE_TIMEOUT with a message.  Over the
    # many barriers of a sweep some CTA is always early.  The context then
    # runs the same sweep normally.
    specs = small_specs(8, seed=12)
    assert any(z2.Lattice(sp["d"], sp["L"]).n_links >= 14 for sp in specs)
    z2.z2_ctx_set_option(ctx, z2.Z2_OPT_GANG_WAIT_POLLS, 1)
    try:
        with pytest.raises(z2.Z2Error) as e:
            z2.z2_sweep(ctx, specs, mode=z2.Z2_SWEEP_PERSISTENT, n_streams=2)
        assert e.value.code == -6
        assert "gave up" in str(e.value)
    finally:
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_GANG_WAIT_POLLS, 0)
    res = z2.z2_sweep(ctx, specs, mode=z2.Z2_SWEEP_PERSISTENT, n_streams=2)
    assert all(r.status == 0 and abs(r.norm - 1) < 1e-5 for r in res)
