"""GPU parity of the densities of states (z2_dos) and of trajectories (runs
measured every k steps) against the FP64 oracle, through the C ABI.

Sec. 3.3 histograms the Z and X terms: Z-DOS bins |psi_i|^2 by the number of
plaquettes with U_p = -1, X-DOS by the number of links with sigma^x = -1 in
the sigma^x basis.  Tolerances as for the other observables: a bin is a
probability (bounded by 1), 1e-5 for complex64 states, 1e-10 for complex128.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1910_08020_gb300 as z2
from oracle.lattice import Lattice as OLattice

pytestmark = pytest.mark.gpu

TOL = {z2.Z2_C64: 1e-5, z2.Z2_C128: 1e-10}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    z2.build()
    c = z2.Context(0)
    yield c.handle
    c.close()


def device_state(psi, precision):
    dt = torch.complex128 if precision == z2.Z2_C128 else torch.complex64
    return torch.from_numpy(psi).to(device="cuda", dtype=dt)


@pytest.mark.parametrize("precision", [z2.Z2_C64, z2.Z2_C128])
@pytest.mark.parametrize("d,L,lam,T,M", [(2, (3, 3), 1.3, 2.0, 12), (2, (2, 2), 2.0, 3.0, 15),
                                         (3, (2, 2, 2), 1.5, 2.0, 6)])
def test_dos_matches_oracle(ctx, precision, d, L, lam, T, M):
    ol = OLattice(d, L)
    psi = oracle.run(ol, lam, T, M, 1)
    lat = z2.Lattice(d, L)
    g = device_state(psi, precision)
    before = g.clone()
    zd = z2.z2_dos(ctx, lat.handle, precision, g, z2.Z2_DOS_Z)
    # the same numbers twice on the same state (fixed-order FP64 reduction)
    assert np.array_equal(zd, z2.z2_dos(ctx, lat.handle, precision, g, z2.Z2_DOS_Z))
    xd = z2.z2_dos(ctx, lat.handle, precision, g, z2.Z2_DOS_X)
    zref = oracle.zdos(psi, ol.plaq_masks())
    xref = oracle.xdos(psi)
    assert zd.shape == (ol.n_plaq + 1,) and xd.shape == (ol.n_links + 1,)
    assert np.max(np.abs(zd - zref)) < TOL[precision], (zd, zref)
    assert np.max(np.abs(xd - xref)) < TOL[precision], (xd, xref)
    # the X density goes through the Hadamard layer and back: state unchanged up to rounding
    assert torch.max(torch.abs(g - before)).item() < (1e-6 if precision == z2.Z2_C64 else 1e-12)


def test_dos_consistent_with_measurement(ctx):
    # sum_k zdos[k] = <psi|psi>, and the first moments reproduce <sum_p U_p> and
    # <sum_l sigma^x_l> from z2_measure (different reductions of the same state)
    d, L, lam, T, M = 2, (4, 3), 3.0, 4.0, 40
    lat = z2.Lattice(d, L)
    n, npq = lat.info.n_links, lat.info.n_plaq
    g = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    p = z2.params(lam, T, M)
    res = z2.results_dict(z2.z2_run(ctx, lat.handle, p, g), lat.info)
    zd = z2.z2_dos(ctx, lat.handle, z2.Z2_C64, g, z2.Z2_DOS_Z)
    xd = z2.z2_dos(ctx, lat.handle, z2.Z2_C64, g, z2.Z2_DOS_X)
    assert abs(zd.sum() - res["norm"]) < 1e-6 and abs(xd.sum() - res["norm"]) < 1e-6
    k = np.arange(npq + 1)
    w = np.arange(n + 1)
    assert abs(((npq - 2 * k) * zd).sum() / zd.sum() - npq * res["mean_plaq"]) < 1e-5
    assert abs(((n - 2 * w) * xd).sum() / xd.sum() - res["sigmax"].sum()) < 1e-5 * n


def test_trajectory_matches_oracle_segments(ctx):
    # every point of the trajectory is the state after j of the M steps, at s = j / M
    d, L, lam, T, M, every = 2, (3, 3), 2.0, 4.0, 20, 6
    ol = OLattice(d, L)
    lat = z2.Lattice(d, L)
    g = torch.empty(1 << ol.n_links, dtype=torch.complex64, device="cuda")
    p = z2.params(lam, T, M)
    pts = z2.trajectory(ctx, lat, p, g, every, dos=True)
    assert [q["step"] for q in pts] == [6, 12, 18, 20]
    psi = oracle.init_plus(ol.n_links)
    j = 0
    S = ol.n_links + lam * ol.n_plaq
    for q in pts:
        oracle.evolve(psi, ol.plaq_masks(), lam, T, M, 1, j0=j, j1=q["step"])
        j = q["step"]
        ref = oracle.observables(ol, psi, lam, s=j / M)
        assert abs(q["energy"] - ref["energy"]) < 1e-5 * S, (j, q["energy"], ref["energy"])
        assert np.max(np.abs(q["plaq"] - ref["plaq"])) < 1e-5
        assert np.max(np.abs(q["zdos"] - oracle.zdos(psi, ol.plaq_masks()))) < 1e-5
        assert np.max(np.abs(q["xdos"] - oracle.xdos(psi))) < 1e-5
    # the last point is the whole run
    whole = z2.results_dict(z2.z2_run(ctx, lat.handle, p, g), lat.info)
    assert abs(whole["energy"] - pts[-1]["energy"]) < 1e-6 * S


def test_dos_rejects_bad_arguments(ctx):
    lat = z2.Lattice(2, (3, 3))
    g = torch.zeros(1 << 18, dtype=torch.complex64, device="cuda")
    with pytest.raises(z2.Z2Error):
        z2.z2_dos(ctx, lat.handle, z2.Z2_C64, g, 7)
    with pytest.raises(z2.Z2Error):
        z2.z2_dos(ctx, lat.handle, 9, g, z2.Z2_DOS_Z)
