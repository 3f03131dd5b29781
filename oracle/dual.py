"""Exact 2+1D duality: Z2 gauge theory <-> transverse-field Ising model.

TEST INFRASTRUCTURE ONLY (see the package docstring).

In two space dimensions the gauge theory is dual to the quantum Ising model
in a transverse field (Sec. 1 and Sec. 3.2).  On the periodic L_x x L_y
lattice, restricted to the sector G_s = 1 (all sites), V_mu = +1, the map

    U_p          <->  tau^x_p                (one dual spin per plaquette)
    sigma^x_l    <->  tau^z_p tau^z_q        (p, q: the two plaquettes of l)

preserves every algebraic relation (each star and each dual loop maps to the
identity, and prod_p U_p = 1 maps to the Z2-even sector prod_p tau^x_p = 1).
It sends |+>^N to (|up...up> + |down...down>)/sqrt(2), each transverse-field
layer R(dt) = prod_l exp(i dt sigma^x_l) to the diagonal bond phase
prod_l exp(i dt tau^z_p tau^z_q) and each plaquette layer D(theta) to
prod_p exp(i theta tau^x_p).  The Trotterised dynamics therefore map step by
step, exactly, onto a 2^{N_p}-dimensional simulation: 16 spins for the
32-link 4x4 lattice.
"""

from __future__ import annotations

import numpy as np

from .ed import lanczos_ground_state
from .lattice import Lattice


class DualIsing:
    def __init__(self, lat: Lattice):
        if lat.d != 2:
            raise ValueError("the gauge/Ising duality used here is 2+1D only")
        self.lat = lat
        self.n = lat.n_plaq
        owners = [[] for _ in range(lat.n_links)]
        for p, links in enumerate(lat.plaq_links):
            for l in links:
                owners[l].append(p)
        assert all(len(o) == 2 for o in owners)
        self.bonds = [tuple(o) for o in owners]  # bond index == link index
        idx = np.arange(1 << self.n, dtype=np.int64)
        self.z = [1.0 - 2.0 * ((idx >> p) & 1) for p in range(self.n)]
        self.bond_zz = [self.z[p] * self.z[q] for p, q in self.bonds]
        self.zz_sum = np.sum(self.bond_zz, axis=0)

    def init_state(self):
        psi = np.zeros(1 << self.n, dtype=np.complex128)
        psi[0] = psi[-1] = 1 / np.sqrt(2.0)
        return psi

    # -- images of the two layers -----------------------------------------------
    def apply_R(self, psi, dt):
        """Image of prod_l exp(i dt sigma^x_l): exp(i dt sum_bonds zz)."""
        psi *= np.exp(1j * dt * self.zz_sum)
        return psi

    def apply_D(self, psi, theta):
        """Image of exp(i theta sum_p U_p): exp(i theta tau^x_p) on each spin."""
        c, s = np.cos(theta), np.sin(theta)
        n = self.n
        for p in range(n):
            v = psi.reshape(1 << (n - p - 1), 2, 1 << p)
            a = v[:, 0, :].copy()
            b = v[:, 1, :].copy()
            v[:, 0, :] = c * a + 1j * s * b
            v[:, 1, :] = 1j * s * a + c * b
        return psi

    def evolve(self, psi, lam, T, M, decomp=1, sampling=0, j0=0, j1=None):
        """Same schedule as the direct oracle (oracle.z2ref_evolve)."""
        dt = T / M
        j1 = M if j1 is None else j1
        for j in range(j0 + 1, j1 + 1):
            s_j, s_jm1 = j / M, (j - 1) / M
            if decomp == 0:
                self.apply_D(psi, lam * s_j * dt)
                self.apply_R(psi, dt)
            else:
                s_first = s_j if sampling else s_jm1
                self.apply_D(psi, lam * s_first * dt / 2)
                self.apply_R(psi, dt)
                self.apply_D(psi, lam * s_j * dt / 2)
        return psi

    def run(self, lam, T, M, decomp=1, sampling=0):
        return self.evolve(self.init_state(), lam, T, M, decomp, sampling)

    # -- observables ------------------------------------------------------------
    def x_expect(self, psi, spins):
        """<prod_{p in spins} tau^x_p> (image of a contractible Wilson loop
        around the plaquettes `spins`)."""
        m = 0
        for p in spins:
            m ^= 1 << p
        idx = np.arange(psi.size)
        return float(np.real(np.vdot(psi[idx ^ m], psi)))

    def observables(self, psi, lam, s=1.0):
        prob = np.abs(psi) ** 2
        sigmax = np.array([float(prob @ zz) for zz in self.bond_zz])
        plaq = np.array([self.x_expect(psi, [p]) for p in range(self.n)])
        lat = self.lat
        out = dict(norm=float(prob.sum()), sigmax=sigmax, plaq=plaq, mean_plaq=plaq.mean(),
                   energy=-sigmax.sum() - s * lam * plaq.sum())
        if lat.L[0] >= 3 and lat.L[1] >= 3:
            ps = [lat.plaquette_index(lat.site([x, y]), 0, 1) for x in (0, 1) for y in (0, 1)]
            out["wilson_2x2"] = self.x_expect(psi, ps)
        else:
            out["wilson_2x2"] = float("nan")
        return out

    # -- ground state -----------------------------------------------------------
    def hamiltonian_apply(self, x, s_lambda):
        """Image of H(s): -sum_bonds zz - s*lambda*sum_p tau^x_p."""
        y = -self.zz_sum * x
        n = self.n
        for p in range(n):
            v = x.reshape(1 << (n - p - 1), 2, 1 << p)
            y -= s_lambda * v[:, ::-1, :].reshape(-1)
        return y

    def ground_state(self, s_lambda, tol=1e-12):
        """Lowest state in the Z2-even sector (the image of the G = 1, V = +
        sector), seeded with the even image of |+>^N."""
        v0 = np.real(self.init_state())
        E, phi, r = lanczos_ground_state(lambda x: self.hamiltonian_apply(x, s_lambda), v0, tol=tol)
        return E, phi.astype(np.complex128), r
