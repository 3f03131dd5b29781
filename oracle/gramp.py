"""The paper's own adiabatic schedule (Sec. 2.2-2.3): TEST INFRASTRUCTURE ONLY,
like the rest of `oracle/`.

The paper ramps H(g) = Z + g X, with Z = sum_p Z_p, Z_p = -prod_{l in p}
sigma^z_l (so Z_p = -U_p) and X = -sum_l sigma^x_l, from g = 0 upward.  Its
start state is the ground state of Z reached by projecting |+>^N onto
Z_p = -1 for every plaquette (Sec. 2.4, "Preparation of the initial ground
state"): the equal superposition of every link configuration with all
U_p = +1, which is also the V_mu = +1 eigenstate.

The ramp has N_s steps of n substeps each; substep m of step k runs for t_s/n
under H_{k,m} = Z + g_{k,m} X with g_{k,m} = (k - 1) g_s + m g_s / n, i.e.
g_j = j g_s / n for the j-th substep overall.  A substep is split
asymmetrically as exp(-i Z t_s/n) exp(-i g X t_s/n) (Eq. a; the X factor acts
first) or symmetrically as exp(-i Z t_s/2n) exp(-i g X t_s/n) exp(-i Z t_s/2n)
(Eq. s).  Measurements are taken at the end of each step, g = k g_s.

In the layer convention of this oracle, D(theta) multiplies amplitude i by
exp(i theta sum_p u_p(i)) and R(a) applies exp(i a sigma^x) to every link, so
exp(-i Z tau) = D(tau) and exp(-i g X tau) = R(g tau): the plaquette angle is
constant and the rotation angle follows the ramp, the reverse of the
H(s) = -sum sigma^x - s lambda sum U_p schedule of the main path.
"""
import numpy as np

from . import FIRST_ORDER, SYMMETRIC, apply_D, apply_R, init_plus, xsums, zsums
from .lattice import Lattice


def _popcount(v):
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(v)
    c = np.zeros(v.shape, dtype=np.uint64)
    for l in range(64):
        c += (v >> np.uint64(l)) & np.uint64(1)
    return c


def init_projected(lat: Lattice) -> np.ndarray:
    """prod_p P_p |+>^N, normalised, with P_p = (1 + U_p) / 2 the projector on
    Z_p = -1 (Sec. 2.4); each projector is applied as written."""
    n = lat.n_links
    psi = init_plus(n)
    idx = np.arange(1 << n, dtype=np.uint64)
    for m in lat.plaq_masks():
        parity = (_popcount(idx & np.uint64(m)) & 1).astype(np.int64)
        u = 1 - 2 * parity
        psi = psi * (1 + u) / 2
    return psi / np.linalg.norm(psi)


def evolve_gramp(psi, lat: Lattice, g_s, t_s, N_s, n, decomp=SYMMETRIC, k0=0, k1=None):
    """Apply steps k0+1 .. k1 (default: to N_s) of the ramp in place, substep by
    substep in the paper's order (Eqs. a and s); decomp is FIRST_ORDER (the
    paper's asymmetric split) or SYMMETRIC."""
    k1 = N_s if k1 is None else k1
    if not (0 <= k0 <= k1 <= N_s) or n < 1:
        raise ValueError("bad ramp arguments")
    masks = lat.plaq_masks()
    tau = t_s / n
    for k in range(k0 + 1, k1 + 1):
        for m in range(1, n + 1):
            g = (k - 1) * g_s + m * g_s / n
            if decomp == FIRST_ORDER:  # the paper's asymmetric split
                apply_R(psi, g * tau)      # exp(-i g X tau), acting first
                apply_D(psi, masks, tau)   # exp(-i Z tau)
            elif decomp == SYMMETRIC:
                apply_D(psi, masks, tau / 2)
                apply_R(psi, g * tau)
                apply_D(psi, masks, tau / 2)
            else:
                raise ValueError("bad decomposition")
    return psi


def energy(lat: Lattice, psi, g):
    """<H(g)> = <Z> + g <X> = -sum_p <U_p> - g sum_l <sigma^x_l> (Sec. 2.4),
    normalised by <psi|psi>."""
    nrm = float(np.vdot(psi, psi).real)
    z = -float(np.sum(zsums(psi, lat.plaq_masks()))) / nrm
    x = -float(np.sum(xsums(psi, [1 << l for l in range(lat.n_links)]).real)) / nrm
    return z + g * x


def _apply_w(psi, lat: Lattice, flips):
    """prod_{mu in flips} W_mu psi, W_mu = prod of sigma^z along the
    non-contractible loop C_mu (diagonal, +-1)."""
    n = lat.n_links
    idx = np.arange(1 << n, dtype=np.uint64)
    w = lat.w_masks()
    out = psi.copy()
    for mu in flips:
        out = out * (1 - 2 * (_popcount(idx & np.uint64(w[mu])) & 1).astype(np.float64))
    return out


def sector_start(lat: Lattice, flips, start=None) -> np.ndarray:
    """A degenerate ground state of Z in another topological sector (Sec. 2.4):
    W_mu applied to the projected start (init_projected(lat), or `start` if
    given) for every mu in `flips`.  W_mu anticommutes with the 't Hooft
    operators V_nu whose surface its loop crosses, so their eigenvalues flip
    from +1 to -1."""
    return _apply_w(init_projected(lat) if start is None else start, lat, flips)


def sector_ground_state(lat: Lattice, g, flips, tol=1e-12):
    """Lowest state of H(g) = Z + gX in the sector of sector_start(lat, flips)
    (Sec. 4.3's E(V_x, V_y, ...)).  H(g) = g (-sum sigma^x - (1/g) sum U_p), so
    this is the Lanczos ground state of the main path's H at s*lambda = 1/g,
    seeded with prod W_mu |+>^N, which lies in that sector (H keeps V_mu and G_s).
    Returns (energy of H(g), state, residual)."""
    from .ed import SparseH, lanczos_ground_state
    n = lat.n_links
    seed = _apply_w(np.full(1 << n, 2.0 ** (-n / 2)), lat, flips)
    E, phi, r = lanczos_ground_state(SparseH(lat, 1.0 / g), seed.real, tol=tol)
    return g * E, phi.astype(np.complex128), r
