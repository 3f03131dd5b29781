"""GPU parity for the gate-level execution (Sec. 2.3, Eq. ara, Figs. 3-4):
each gate kernel against the oracle's gates, and the paper's ramp run gate by
gate with the ancilla circuit for every plaquette factor against the fused
FP64 oracle (oracle/gramp.py), with the paper's gate count per substep
(N + 9 N_p: 99 on the 3x3 lattice, 240 on 2x2x2).

Tolerances: one gate 1e-6 (complex64) / 1e-13 (complex128) of the largest
amplitude; a ramp 1e-5 / 1e-10; the ancilla's |1> half stays below the same.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1910_08020_gb300 as z2
from oracle import gramp
from oracle.circuit import _cnot, _rz
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
@pytest.mark.parametrize("n", [9, 13])
def test_single_gates_match_oracle(ctx, n, precision):
    tol = 1e-13 if precision == z2.Z2_C128 else 1e-6
    psi = workloads.random_state(n, seed=n)
    rng = np.random.default_rng(n)
    for _ in range(6):
        c, t = (int(x) for x in rng.choice(n, size=2, replace=False))
        g = dev(psi, precision)
        z2.z2_apply_gate(ctx, n, precision, g, z2.Z2_GATE_CNOT, c, t)
        assert rel_err(host(g), _cnot(psi, c, t)) < tol
        q, phi = int(rng.integers(n)), float(rng.uniform(-4, 4))
        g = dev(psi, precision)
        z2.z2_apply_gate(ctx, n, precision, g, z2.Z2_GATE_RZ, q, -1, phi)
        assert rel_err(host(g), _rz(psi, q, phi)) < tol
        g = dev(psi, precision)
        z2.z2_apply_gate(ctx, n, precision, g, z2.Z2_GATE_RX, q, -1, phi)
        # R_x(phi) = exp(-i phi sigma^x / 2) = the oracle's exp(i dt sigma^x) at dt = -phi/2
        assert rel_err(host(g), oracle.apply_rx(psi.copy(), q, -phi / 2)) < tol
    g = dev(psi, precision)
    for q in range(n):
        z2.z2_apply_gate(ctx, n, precision, g, z2.Z2_GATE_H, q)
    assert rel_err(host(g), oracle.apply_hadamard_all(psi.copy())) < tol


def test_gate_argument_errors(ctx):
    g = torch.zeros(1 << 9, dtype=torch.complex64, device="cuda")
    for args in ((z2.Z2_GATE_CNOT, 3, 3), (z2.Z2_GATE_RZ, 9, -1), (7, 0, -1)):
        with pytest.raises(z2.Z2Error):
            z2.z2_apply_gate(ctx, 9, z2.Z2_C64, g, *args, 0.3)


@pytest.mark.parametrize("precision", [z2.Z2_C64, z2.Z2_C128])
@pytest.mark.parametrize("decomp", [z2.Z2_FIRST_ORDER, z2.Z2_SYMMETRIC])
@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3))])
def test_ramp_gate_by_gate_matches_fused_oracle(ctx, d, L, decomp, precision):
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    N, Np = ol.n_links, ol.n_plaq
    g_s, t_s, N_s, n = 0.3, 0.6, 2, 3
    gp = z2.gramp_params(g_s, t_s, N_s, n, decomp, precision)
    dt = torch.complex128 if precision == z2.Z2_C128 else torch.complex64
    g = torch.zeros(2 << N, dtype=dt, device="cuda")
    z2.z2_init_projected(ctx, lat.handle, precision, g)  # the links' half; the ancilla (bit N) in |0>
    gates = z2.z2_evolve_gramp_circuit(ctx, lat.handle, gp, g, 0, N_s)
    per_sub = N + (18 if decomp == z2.Z2_SYMMETRIC else 9) * Np
    assert gates == N_s * n * per_sub
    want = gramp.evolve_gramp(gramp.init_projected(ol), ol, g_s, t_s, N_s, n, decomp)
    got = host(g)
    tol = 1e-10 if precision == z2.Z2_C128 else 1e-5
    assert rel_err(got[: 1 << N], want) < tol
    assert np.max(np.abs(got[1 << N:])) < tol  # the ancilla is back in |0>
    # and the fused passes give the same links' state
    f = torch.empty(1 << N, dtype=dt, device="cuda")
    z2.z2_run_gramp(ctx, lat.handle, gp, f)
    assert rel_err(host(f), got[: 1 << N]) < tol


def test_paper_gate_counts_per_substep(ctx):
    # Sec. 2.3 and 2.6: one substep of the asymmetric split takes N_l gates for
    # the transverse field and 9 per plaquette (4 CNOT, R_z, 4 CNOT)
    for d, L, per_sub in ((2, (3, 3), 18 + 9 * 9), (3, (2, 2, 2), 24 + 9 * 24)):
        lat = z2.Lattice(d, L)
        N = lat.n_links
        g = torch.zeros(2 << N, dtype=torch.complex64, device="cuda")
        gp = z2.gramp_params(0.1, 0.1, 1, 1, z2.Z2_FIRST_ORDER, z2.Z2_C64)
        assert z2.z2_evolve_gramp_circuit(ctx, lat.handle, gp, g, 0, 1) == per_sub
