"""GPU parity for the controlled evolution of phase estimation (Sec. 2.4,
Eq. leap, Fig. 5): U(t) = |0><0| (x) exp(-iHt) + |1><1| (x) exp(iHt) for
H = Z + g X at fixed g, on the fused passes, against the FP64 oracle
(oracle/qpe.py); the phase read out from an eigenstate against 2 E t within
the paper's Trotter error estimate; time reversal of the symmetric formula.

Tolerances: complex64 1e-5 of the largest amplitude, complex128 1e-10.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1910_08020_gb300 as z2
from oracle import gramp, qpe
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


def dev(psi, precision):
    dt = torch.complex128 if precision == z2.Z2_C128 else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(psi)).to(dt).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", [z2.Z2_C64, z2.Z2_C128])
@pytest.mark.parametrize("decomp", [z2.Z2_FIRST_ORDER, z2.Z2_SYMMETRIC])
@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3)), (2, (4, 2))])
def test_controlled_evolution_matches_oracle(ctx, d, L, decomp, precision):
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    psi = workloads.random_state(ol.n_links + 1, seed=21)
    g = dev(psi, precision)
    z2.z2_controlled_evolution(ctx, lat.handle, z2.qpe_params(0.8, 1.1, 9, decomp, precision), g)
    want = qpe.controlled_evolution(psi.copy(), ol, 0.8, 1.1, 9, decomp)
    assert rel_err(host(g), want) < (1e-10 if precision == z2.Z2_C128 else 1e-5)


def test_phase_of_an_eigenstate_3x3(ctx):
    # the ground state u of H(g) = Z + g X in the gauge sector (oracle Lanczos),
    # with the control in (|0> + |1>)/sqrt(2): <half 0|half 1> = e^{2iEt}/2,
    # for t = 2^k t0 as phase estimation needs
    lat = z2.Lattice(2, (3, 3))
    ol = OLattice(2, (3, 3))
    N = ol.n_links
    g_c, t0, n = 0.5, 0.25, 40
    E, u, r = gramp.sector_ground_state(ol, g_c, [])
    assert r < 1e-9
    base = np.concatenate([u, u]) / np.sqrt(2)
    for k in range(4):
        t = t0 * 2 ** k
        g = dev(base, z2.Z2_C128)
        z2.z2_controlled_evolution(ctx, lat.handle, z2.qpe_params(g_c, t, n * 2 ** k, z2.Z2_SYMMETRIC, z2.Z2_C128), g)
        half = 16 << N  # bytes of one complex128 branch
        c = z2.z2_overlap(ctx, N, z2.Z2_C128, g.data_ptr(), g.data_ptr() + half)
        want = qpe.controlled_evolution(base.copy(), ol, g_c, t, n * 2 ** k, z2.Z2_SYMMETRIC)
        assert abs(c - qpe.ancilla_coherence(want, N)) < 1e-10
        bound = ((2 - 1) * g_c + 4 * g_c ** 2) / 3 * ol.n_plaq * t ** 3 / (n * 2 ** k) ** 2
        assert abs(c - np.exp(2j * E * t) / 2) <= bound


def test_symmetric_controlled_evolution_reverses(ctx):
    lat = z2.Lattice(2, (3, 3))
    psi = workloads.random_state(19, seed=5)
    g = dev(psi, z2.Z2_C64)
    z2.z2_controlled_evolution(ctx, lat.handle, z2.qpe_params(1.3, 0.7, 11, z2.Z2_SYMMETRIC, z2.Z2_C64), g)
    z2.z2_controlled_evolution(ctx, lat.handle, z2.qpe_params(1.3, -0.7, 11, z2.Z2_SYMMETRIC, z2.Z2_C64), g)
    assert rel_err(host(g), psi) < 1e-5


def test_controlled_evolution_argument_errors(ctx):
    lat = z2.Lattice(2, (2, 2))
    g = torch.zeros(1 << 9, dtype=torch.complex64, device="cuda")
    for qp in (z2.qpe_params(1, 1, 0), z2.qpe_params(1, 1, 3, decomp=4), z2.qpe_params(1, float("nan"), 3)):
        with pytest.raises(z2.Z2Error):
            z2.z2_controlled_evolution(ctx, lat.handle, qp, g)
