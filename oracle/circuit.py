"""The paper's gate-level realisation of the plaquette factors (Sec. 2.3,
Eq. ara and Fig. 3): TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`.

exp(-i Z_p tau) = A^-1 R_z^a(-2 tau) A, where A is the four CNOTs from the
plaquette's links onto one ancilla qubit a (initially |0>) and
R_z(phi) = exp(-i sigma^z phi / 2).  The ancilla ends up holding the
plaquette's parity, the rotation gives exp(+i tau) for even and exp(-i tau)
for odd parity, and the second set of CNOTs returns the ancilla to |0>.
Here the N link qubits are index bits 0..N-1 and the ancilla is bit N.
"""
import numpy as np


def _cnot(psi, control, target):
    """CNOT on a state vector: flip `target` where `control` is 1."""
    idx = np.arange(len(psi), dtype=np.uint64)
    sel = ((idx >> np.uint64(control)) & np.uint64(1)).astype(bool)
    out = psi.copy()
    out[sel] = psi[(idx ^ (np.uint64(1) << np.uint64(target)))[sel]]
    return out


def _rz(psi, qubit, phi):
    idx = np.arange(len(psi), dtype=np.uint64)
    bit = ((idx >> np.uint64(qubit)) & np.uint64(1)).astype(np.int64)
    return psi * np.exp(-1j * phi / 2 * (1 - 2 * bit))


def apply_plaquettes_with_ancilla(psi_links, plaq_masks, tau):
    """prod_p exp(-i Z_p tau) on an N-link state, gate by gate through one
    ancilla as in Fig. 3.  Returns (the N-link state, the largest amplitude
    left with the ancilla in |1>, which the circuit keeps at zero)."""
    n = int(np.log2(len(psi_links)))
    psi = np.concatenate([psi_links, np.zeros_like(psi_links)])  # ancilla (bit n) in |0>
    for m in plaq_masks:
        links = [l for l in range(n) if (int(m) >> l) & 1]
        for l in links:
            psi = _cnot(psi, l, n)
        psi = _rz(psi, n, -2.0 * tau)
        for l in reversed(links):
            psi = _cnot(psi, l, n)
    return psi[: 1 << n], float(np.max(np.abs(psi[1 << n:])))
