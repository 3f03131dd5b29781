"""Full-size GPU parity at the paper-shaped workloads, against the exact 2+1D
gauge/Ising duality (oracle/dual.py), which maps the Trotterised dynamics
step by step onto 2^{N_p}-dimensional spin simulations:

  4x3 periodic, 24 qubits  <->  12 dual spins
  4x4 periodic, 32 qubits  <->  16 dual spins   (34.4 GB complex64 state)

lambda = 3, T = 20, M = 500, first order and symmetric, complex64 state,
the same launch configuration the benchmark times.  Fidelity is against the
dual ground state lifted to the link basis (sigma^x basis amplitudes
sqrt(2) phi(tau) on the configurations x_l = tau_p tau_q).  The 24-qubit
case is also checked against the direct FP64 state-vector oracle.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1910_08020_gb300 as z2
from oracle.dual import DualIsing
from oracle.lattice import Lattice as OLattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    z2.build()
    c = z2.Context(0)
    yield c.handle
    c.close()


def xbasis_index(ol, du):
    """Link sigma^x-basis index of every dual configuration tau."""
    n = du.n
    taus = np.arange(1 << n, dtype=np.int64)
    idx = np.zeros(1 << n, dtype=np.int64)
    for l, (p, q) in enumerate(du.bonds):
        flip = ((taus >> p) ^ (taus >> q)) & 1  # tau_p tau_q = -1
        idx |= flip << l
    return idx


@pytest.mark.parametrize("L,decomp", [((4, 3), 1), ((4, 3), 0), ((4, 4), 1), ((4, 4), 0)])
def test_against_dual(ctx, L, decomp):
    lam, T, M = 3.0, 20.0, 500
    ol = OLattice(2, L)
    du = DualIsing(ol)
    psi_d = du.run(lam, T, M, decomp)
    ref = du.observables(psi_d, lam)
    E0, phi_d, r = du.ground_state(lam)
    assert r < 1e-10
    F_ref = abs(np.vdot(phi_d, psi_d)) ** 2

    lat = z2.Lattice(2, L)
    n = ol.n_links
    g = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    res = z2.z2_run(ctx, lat.handle, z2.params(lam, T, M, decomp, z2.Z2_C64), g)
    d = z2.results_dict(res, lat.info)
    S = n + lam * ol.n_plaq
    assert abs(d["energy"] - ref["energy"]) < 1e-5 * S, (d["energy"], ref["energy"])
    assert np.max(np.abs(d["plaq"] - ref["plaq"])) < 1e-5
    assert np.max(np.abs(d["sigmax"] - ref["sigmax"])) < 1e-5
    assert abs(d["wilson_2x2"] - ref["wilson_2x2"]) < 1e-5
    assert abs(d["norm"] - 1) < 1e-5
    assert np.max(np.abs(d["star"] - 1)) < 1e-5
    assert np.max(np.abs(d["sigmaz"])) < 1e-5

    # fidelity with the ground state: overlap in the sigma^x basis
    z2.z2_apply_hadamard(ctx, lat.handle, z2.Z2_C64, g)
    idx = xbasis_index(ol, du)
    xs = torch.from_numpy(idx).cuda()
    psi_x = g[xs].cpu().numpy().astype(np.complex128)
    # each x configuration arises from tau and -tau: sum over tau / 2 with weight sqrt(2) phi(tau)
    ov = np.sum(np.conj(np.sqrt(2.0) * phi_d) * psi_x) / 2.0
    F = abs(ov) ** 2 / d["norm"]
    assert abs(F - F_ref) < 1e-6, (F, F_ref, d["norm"], abs(ov) ** 2)
    del g
    torch.cuda.empty_cache()


@pytest.mark.parametrize("decomp", [1, 0])
def test_24_qubit_subcase_against_direct_oracle(ctx, decomp):
    # the 32-qubit configuration's 24-qubit sub-case (4x3, lambda = 3, T = 20,
    # M = 500, both splits) against the direct FP64 state-vector oracle, not
    # only through the duality: every observable, and the state's fidelity
    # loss (<= 1e-6)
    lam, T, M = 3.0, 20.0, 500
    ol = OLattice(2, (4, 3))
    psi = oracle.run(ol, lam, T, M, decomp)
    ref = oracle.observables(ol, psi, lam)
    lat = z2.Lattice(2, (4, 3))
    g = torch.empty(1 << 24, dtype=torch.complex64, device="cuda")
    res = z2.z2_run(ctx, lat.handle, z2.params(lam, T, M, decomp, z2.Z2_C64), g)
    d = z2.results_dict(res, lat.info)
    S = ol.n_links + lam * ol.n_plaq
    assert abs(d["energy"] - ref["energy"]) < 1e-5 * S
    for k in ("plaq", "sigmax", "sigmaz", "star", "wmu", "vmu"):
        assert np.max(np.abs(d[k] - ref[k])) < 1e-5, k
    assert abs(d["wilson_2x2"] - ref["wilson_2x2"]) < 1e-5
    torch.cuda.synchronize()
    got = g.cpu().numpy().astype(np.complex128)
    f = abs(np.vdot(psi, got)) ** 2 / (np.vdot(psi, psi).real * np.vdot(got, got).real)
    assert 1 - f < 1e-6, 1 - f
