"""FP64 CPU oracle for the Z2 lattice-gauge-theory adiabatic state-vector path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library and never imports it.

Contents
  lattice.py  independent lattice builder (links, plaquettes, stars, loops)
  z2ref.c     plain FP64 state-vector simulator: |+>, D(theta), R(dt), the
              first-order and symmetric steps, sigma^z/sigma^x-type sums
  ed.py       dense exact diagonalisation, Lanczos, 4th-order Magnus reference
  dual.py     the exact 2+1D gauge <-> transverse-field Ising duality simulator

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, brute force, library routines or the exact duality.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

from .lattice import Lattice  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libz2ref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile z2ref.c with the host C compiler (plain C99 + OpenMP)."""
    src = os.path.join(_HERE, "z2ref.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        up = ctypes.POINTER(ctypes.c_uint64)
        i, d = ctypes.c_int, ctypes.c_double
        L.z2ref_init_plus.argtypes = [i, dp]
        L.z2ref_apply_D.argtypes = [i, dp, i, up, d]
        L.z2ref_apply_rx_qubit.argtypes = [i, dp, i, d]
        L.z2ref_apply_R.argtypes = [i, dp, d]
        L.z2ref_apply_hadamard_all.argtypes = [i, dp]
        L.z2ref_evolve.argtypes = [i, dp, i, up, d, d, i, i, i, i, i]
        L.z2ref_evolve.restype = ctypes.c_int
        L.z2ref_zsums.argtypes = [i, dp, i, up, dp]
        L.z2ref_xsums.argtypes = [i, dp, i, up, dp]
        L.z2ref_zdos.argtypes = [i, dp, i, up, dp]
        L.z2ref_overlap.argtypes = [i, dp, dp, dp]
        L.z2ref_hamiltonian_apply.argtypes = [i, dp, dp, i, up, d]
        _lib = L
    return _lib


def _dp(a):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _rp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _up(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _n_of(psi):
    n = int(psi.size).bit_length() - 1
    assert psi.size == 1 << n
    return n


FIRST_ORDER, SYMMETRIC = 0, 1
SAMPLE_STD, SAMPLE_PAPER = 0, 1


# -- primitive operators ------------------------------------------------------
def init_plus(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().z2ref_init_plus(n, _dp(psi))
    return psi


def apply_D(psi, plaq_masks, theta):
    m, mp = _up(plaq_masks)
    lib().z2ref_apply_D(_n_of(psi), _dp(psi), len(m), mp, float(theta))
    return psi


def apply_rx(psi, l, dt):
    lib().z2ref_apply_rx_qubit(_n_of(psi), _dp(psi), int(l), float(dt))
    return psi


def apply_R(psi, dt):
    lib().z2ref_apply_R(_n_of(psi), _dp(psi), float(dt))
    return psi


def apply_hadamard_all(psi):
    lib().z2ref_apply_hadamard_all(_n_of(psi), _dp(psi))
    return psi


def evolve(psi, plaq_masks, lam, T, M, decomp=SYMMETRIC, sampling=SAMPLE_STD, j0=0, j1=None):
    """Apply steps j0+1..j1 of the M-step schedule in place (see z2ref.c)."""
    m, mp = _up(plaq_masks)
    j1 = M if j1 is None else j1
    rc = lib().z2ref_evolve(_n_of(psi), _dp(psi), len(m), mp, float(lam), float(T), int(M),
                            int(decomp), int(sampling), int(j0), int(j1))
    if rc != 0:
        raise ValueError("bad schedule arguments")
    return psi


def run(lat: Lattice, lam, T, M, decomp=SYMMETRIC, sampling=SAMPLE_STD):
    psi = init_plus(lat.n_links)
    return evolve(psi, lat.plaq_masks(), lam, T, M, decomp, sampling)


# -- observables ----------------------------------------------------------------
def zsums(psi, masks):
    m, mp = _up(masks)
    out = np.zeros(len(m), dtype=np.float64)
    if len(m):
        lib().z2ref_zsums(_n_of(psi), _dp(psi), len(m), mp, _rp(out))
    return out


def xsums(psi, masks):
    m, mp = _up(masks)
    out = np.zeros(2 * len(m), dtype=np.float64)
    if len(m):
        lib().z2ref_xsums(_n_of(psi), _dp(psi), len(m), mp, _rp(out))
    return out[0::2] + 1j * out[1::2]


def zdos(psi, plaq_masks):
    m, mp = _up(plaq_masks)
    out = np.zeros(len(m) + 1, dtype=np.float64)
    lib().z2ref_zdos(_n_of(psi), _dp(psi), len(m), mp, _rp(out))
    return out


def xdos(psi):
    """Distribution of the number w of links with sigma^x = -1 (Sec. 3.3;
    X = -sum sigma^x = 2w - N): transform to the sigma^x basis with a Hadamard
    on every qubit, then bin |amplitude|^2 by the number of set bits."""
    phi = apply_hadamard_all(psi.copy())
    n = _n_of(psi)
    idx = np.arange(1 << n, dtype=np.uint64)
    w = np.zeros(1 << n, dtype=np.int64)
    for l in range(n):
        w += ((idx >> np.uint64(l)) & np.uint64(1)).astype(np.int64)
    return np.bincount(w, weights=np.abs(phi) ** 2, minlength=n + 1)


def overlap(a, b):
    out = np.zeros(2, dtype=np.float64)
    lib().z2ref_overlap(_n_of(a), _dp(a), _dp(b), _rp(out))
    return complex(out[0], out[1])


def hamiltonian_apply(lat: Lattice, x, s_lambda):
    y = np.empty_like(x)
    m, mp = _up(lat.plaq_masks())
    lib().z2ref_hamiltonian_apply(lat.n_links, _dp(x), _dp(y), len(m), mp, float(s_lambda))
    return y


def observables(lat: Lattice, psi, lam, s=1.0, ref=None):
    """All end-of-run quantities, each from its plain definition (Sec. 2.4).

    energy      <H(s)> = -sum_l <sigma^x_l> - s*lam*sum_p <U_p>
    plaq[p]     <U_p>, mean_plaq their mean
    wilson_2x2  <W> of the 2x2 loop at the origin (NaN when degenerate)
    contours    <W_c1>, <W_c2>, <W_c3>  (NaN when degenerate)
    star[s]     <G_s>, mean_star their mean (Gauss law)
    sigmaz[l], sigmax[l], wmu[mu], vmu[mu], zdos[k], norm, fidelity
    """
    pm = lat.plaq_masks()
    plaq = zsums(psi, pm)
    sx = xsums(psi, np.array([1 << l for l in range(lat.n_links)], dtype=np.uint64)).real
    star = xsums(psi, lat.star_masks()).real
    w2, w2deg = lat.wilson_2x2()
    cont = lat.contours()
    zm = np.array([0, w2] + [c[0] for c in cont] + list(lat.w_masks())
                  + [1 << l for l in range(lat.n_links)], dtype=np.uint64)
    z = zsums(psi, zm)
    norm = z[0]
    wil = z[1] if not w2deg else float("nan")
    cvals = [z[2 + k] if not cont[k][1] else float("nan") for k in range(3)]
    wmu = z[5:5 + lat.d]
    sigmaz = z[5 + lat.d:]
    vmu = xsums(psi, lat.v_masks()).real
    out = dict(
        norm=norm,
        energy=-sx.sum() - s * lam * plaq.sum(),
        plaq=plaq, mean_plaq=plaq.mean(),
        wilson_2x2=wil, contours=np.array(cvals),
        star=star, mean_star=star.mean(),
        sigmaz=sigmaz, sigmax=sx, wmu=wmu, vmu=vmu,
        zdos=zdos(psi, pm),
    )
    if ref is not None:
        out["fidelity"] = abs(overlap(ref, psi)) ** 2
    return out
