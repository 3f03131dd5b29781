"""Exact diagonalisation, Lanczos and an accurate time-ordered reference
evolution for small Z2 gauge lattices (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Hamiltonian ramped by the adiabatic run (the "start from the ground state of
X, H = X + K Z" variant of Sec. 2.3, with K = s*lambda):

    H(s) = -sum_l sigma^x_l - s*lambda*sum_p U_p,   U_p = prod_{l in p} sigma^z_l
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from .lattice import Lattice


def plaquette_diagonal(lat: Lattice) -> np.ndarray:
    """sum_p U_p on every basis state, from the definition (Sec. 2.1)."""
    n = lat.n_links
    idx = np.arange(1 << n, dtype=np.uint64)
    tot = np.zeros(1 << n, dtype=np.float64)
    for m in lat.plaq_masks():
        par = np.zeros(1 << n, dtype=np.uint64)
        v = idx & np.uint64(m)
        while True:
            nz = v != 0
            if not nz.any():
                break
            par ^= (v & np.uint64(1))
            v = v >> np.uint64(1)
        tot += 1.0 - 2.0 * par.astype(np.float64)
    return tot


def hamiltonian_dense(lat: Lattice, s_lambda: float) -> np.ndarray:
    """Dense real symmetric H(s) (n_links <= 12)."""
    n = lat.n_links
    if n > 12:
        raise ValueError("dense H limited to 12 qubits")
    dim = 1 << n
    H = np.diag(-s_lambda * plaquette_diagonal(lat))
    rows = np.arange(dim)
    for l in range(n):
        H[rows ^ (1 << l), rows] -= 1.0
    return H


class SparseH:
    """Matrix-free real H(s) for Lanczos: sigma^x_l flips bit l."""

    def __init__(self, lat: Lattice, s_lambda: float):
        self.n = lat.n_links
        self.diag = -s_lambda * plaquette_diagonal(lat)

    def __call__(self, x):
        n = self.n
        y = self.diag * x
        for l in range(n):
            v = x.reshape(1 << (n - l - 1), 2, 1 << l)
            y -= v[:, ::-1, :].reshape(-1)
        return y


def lanczos_ground_state(matvec, v0, tol=1e-11, krylov=60, max_restarts=200):
    """Lowest eigenpair of a real symmetric operator by restarted Lanczos with
    full reorthogonalisation, seeded by v0 (the symmetry sector of v0 is kept
    because H maps it into itself).  Returns (E0, phi0, residual)."""
    v = np.asarray(v0, dtype=np.float64).copy()
    v /= np.linalg.norm(v)
    E = None
    for _ in range(max_restarts):
        V = [v]
        alpha, beta = [], []
        w = matvec(v)
        for k in range(krylov):
            a = float(V[k] @ w)
            alpha.append(a)
            w = w - a * V[k] - (beta[-1] * V[k - 1] if k > 0 else 0.0)
            for u in V:  # full reorthogonalisation
                w -= (u @ w) * u
            b = float(np.linalg.norm(w))
            if b < 1e-13 or k == krylov - 1:
                break
            beta.append(b)
            V.append(w / b)
            w = matvec(V[-1])
        Tm = np.diag(alpha) + np.diag(beta[:len(alpha) - 1], 1) + np.diag(beta[:len(alpha) - 1], -1)
        evals, evecs = np.linalg.eigh(Tm)
        E = float(evals[0])
        y = evecs[:, 0]
        v = sum(c * u for c, u in zip(y, V))
        v /= np.linalg.norm(v)
        r = float(np.linalg.norm(matvec(v) - E * v))
        if r < tol:
            return E, v, r
    return E, v, r


def ground_state(lat: Lattice, s_lambda: float, tol=1e-11):
    """Ground state of H(s) in the (G = 1, V = +) sector, seeded with |+>^N
    (which lies in that sector; for s*lambda > 0 it holds the ground state,
    Sec. 2.1).  Returns (E0, phi0 as complex128, residual)."""
    n = lat.n_links
    v0 = np.full(1 << n, 2.0 ** (-n / 2))
    E, phi, r = lanczos_ground_state(SparseH(lat, s_lambda), v0, tol=tol)
    return E, phi.astype(np.complex128), r


def magnus4_evolution(lat: Lattice, lam: float, T: float, steps: int, psi0=None):
    """Time-ordered evolution psi(T) = Texp(-i int_0^T H(t/T) dt) psi(0) by the
    4th-order Magnus integrator with two Gauss-Legendre nodes per step:
        Omega = -i h/2 (H1 + H2) - (sqrt(3)/12) h^2 [H2, H1]
    applied with a dense matrix exponential (n_links <= 12).  This is the
    "exact" evolution that Trotter schemes approximate."""
    n = lat.n_links
    H0 = hamiltonian_dense(lat, 0.0)
    P = -plaquette_diagonal(lat)  # H(s) = H0 + s*lam*diag(P)
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128) if psi0 is None else psi0.copy()
    h = T / steps
    c1, c2 = 0.5 - math.sqrt(3) / 6, 0.5 + math.sqrt(3) / 6
    for k in range(steps):
        H1 = H0 + np.diag(lam * ((k + c1) * h / T) * P)
        H2 = H0 + np.diag(lam * ((k + c2) * h / T) * P)
        Om = -0.5j * h * (H1 + H2) - (math.sqrt(3) / 12.0) * h * h * (H2 @ H1 - H1 @ H2)
        psi = scipy.linalg.expm(Om) @ psi
    return psi
