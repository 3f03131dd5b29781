"""GPU parity: every kernel and whole runs through the C ABI against the FP64
oracle, element by element on seeded random states and on the paper's
workloads (3x3 lattice, 18 qubits; 2x2x2, 24 qubits; 4x3, 24 qubits).

Tolerances, from the arithmetic: the state is complex64 with angles, phase
tables and reductions in FP64, so each layer rounds each amplitude a few
times in FP32 (about 24 rotation levels x 2^-24 = 1.4e-6 relative):
  complex64 layers: max|gpu - ref| <= 2e-6 * max|ref| per layer
  complex64 runs: observables |a - b| <= 1e-5 * S, S = 1 for bounded
    observables and N + lambda N_p for the energy; fidelity 1e-6
  complex128: 1e-10 (layers 1e-12)
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1910_08020_gb300 as z2
from oracle import ed
from oracle.lattice import Lattice as OLattice
from paper_1910_08020_gb300 import workloads

pytestmark = pytest.mark.gpu

LAT_BY_N = {8: (2, (2, 2)), 12: (2, (3, 2)), 16: (2, (4, 2)), 18: (2, (3, 3)), 20: (2, (5, 2)), 24: (2, (4, 3))}


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
    t = torch.from_numpy(np.ascontiguousarray(psi)).to(dt).cuda()
    assert t.data_ptr() % 256 == 0
    return t


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def layer_tol(precision):
    return 1e-12 if precision == z2.Z2_C128 else 2e-6


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


PRECS = [z2.Z2_C64, z2.Z2_C128]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n", [8, 12, 16, 18, 20, 24])
@pytest.mark.parametrize("dt", [0.037, -0.61, 1.3, 2.9])
def test_rx_layer(ctx, n, precision, dt):
    d, L = LAT_BY_N[n]
    lat = z2.Lattice(d, L)
    psi = workloads.random_state(n, seed=100 + n)
    g = dev(psi, precision)
    z2.z2_apply_rx_layer(ctx, lat.handle, precision, g, dt)
    ref = oracle.apply_R(psi.copy(), dt)
    assert rel_err(host(g), ref) < layer_tol(precision)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 3)), (2, (5, 2)), (3, (2, 2, 2)), (2, (4, 3))])
def test_plaquette_layer(ctx, d, L, precision):
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    psi = workloads.random_state(ol.n_links, seed=7)
    for theta in (0.0123, -0.75):
        g = dev(psi, precision)
        z2.z2_apply_plaquettes(ctx, lat.handle, precision, g, theta)
        ref = oracle.apply_D(psi.copy(), ol.plaq_masks(), theta)
        assert rel_err(host(g), ref) < layer_tol(precision)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n", [8, 16, 18, 24])
def test_hadamard_layer(ctx, n, precision):
    d, L = LAT_BY_N[n]
    lat = z2.Lattice(d, L)
    psi = workloads.random_state(n, seed=5)
    g = dev(psi, precision)
    z2.z2_apply_hadamard(ctx, lat.handle, precision, g)
    ref = oracle.apply_hadamard_all(psi.copy())
    assert rel_err(host(g), ref) < layer_tol(precision)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n", [8, 12, 13, 14, 18, 24])
def test_zsums_and_overlap(ctx, n, precision):
    # n < 13: run-based kernel; n >= 13: chunked Walsh-Hadamard kernel (one
    # block at 13 qubits); 42 + n masks = two launches of up to 64 masks
    psi = workloads.random_state(n, seed=9)
    phi = workloads.random_state(n, seed=10)
    rng = np.random.default_rng(n)
    masks = np.concatenate([[0], rng.integers(0, 1 << n, size=40, dtype=np.uint64),
                            [1 << l for l in range(n)]]).astype(np.uint64)
    g = dev(psi, precision)
    got = z2.z2_zsums(ctx, n, precision, g, masks)
    psi_r = host(g)  # the device copy (rounded to the state's precision)
    want = oracle.zsums(psi_r, masks)
    tol = 1e-12 if precision == z2.Z2_C128 else 1e-6
    assert np.max(np.abs(got - want)) < tol
    h = dev(phi, precision)
    ov = z2.z2_overlap(ctx, n, precision, h, g)
    want = oracle.overlap(host(h), psi_r)
    assert abs(ov - want) < tol


def obs_tol(precision, lat, lam):
    base = 1e-10 if precision == z2.Z2_C128 else 1e-5
    return base, base * (lat.n_links + abs(lam) * lat.n_plaq)


def compare_obs(res, ref, lat, lam, precision, with_fid=False):
    d = z2.results_dict(res, lat.info)
    t, tE = obs_tol(precision, lat, lam)
    assert abs(d["norm"] - ref["norm"]) < t
    assert abs(d["energy"] - ref["energy"]) < tE, (d["energy"], ref["energy"])
    assert np.max(np.abs(d["plaq"] - ref["plaq"])) < t
    assert np.max(np.abs(d["sigmax"] - ref["sigmax"])) < t
    assert np.max(np.abs(d["sigmaz"] - ref["sigmaz"])) < t
    assert np.max(np.abs(d["star"] - ref["star"])) < t
    assert np.max(np.abs(d["wmu"] - ref["wmu"])) < t
    assert np.max(np.abs(d["vmu"] - ref["vmu"])) < t
    if math.isnan(ref["wilson_2x2"]):
        assert math.isnan(d["wilson_2x2"]) and d["flags"] & z2.Z2_FLAG_WILSON_DEGENERATE
    else:
        assert abs(d["wilson_2x2"] - ref["wilson_2x2"]) < t
    for k in range(3):
        if math.isnan(ref["contours"][k]):
            assert math.isnan(d["contours"][k])
        else:
            assert abs(d["contours"][k] - ref["contours"][k]) < t
    if with_fid:
        ft = 1e-10 if precision == z2.Z2_C128 else 1e-6
        assert abs(d["fidelity"] - ref["fidelity"]) < ft, (d["fidelity"], ref["fidelity"])
    return d


@pytest.mark.parametrize("precision", PRECS)
def test_config1_3x3_symmetric_with_fidelity(ctx, precision):
    # 3x3 periodic, 18 qubits, lambda = 1, T = 10, M = 200 symmetric, |+>^18
    d, L, lam, T, M = 2, (3, 3), 1.0, 10.0, 200
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    E0, phi0, r = ed.ground_state(ol, lam)
    assert r < 1e-9
    psi = oracle.run(ol, lam, T, M, 1)
    ref = oracle.observables(ol, psi, lam, ref=phi0)
    g = torch.empty(1 << ol.n_links, dtype=torch.complex128 if precision else torch.complex64, device="cuda")
    ref_dev = dev(phi0, precision)
    p = z2.params(lam, T, M, z2.Z2_SYMMETRIC, precision)
    res = z2.z2_run(ctx, lat.handle, p, g, ref=ref_dev)
    compare_obs(res, ref, lat, lam, precision, with_fid=True)
    # the final state itself, amplitude by amplitude
    assert rel_err(host(g), psi) < (1e-10 if precision else 2e-5)


@pytest.mark.parametrize("decomp,sampling", [(0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("d,L", [(2, (2, 2)), (2, (3, 2)), (2, (4, 2)), (2, (3, 3)), (2, (5, 2))])
def test_runs_small_lattices(ctx, d, L, decomp, sampling):
    lam, T, M = 2.7, 3.0, 37
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    psi = oracle.run(ol, lam, T, M, decomp, sampling)
    ref = oracle.observables(ol, psi, lam)
    for precision in PRECS:
        g = torch.empty(1 << ol.n_links, dtype=torch.complex128 if precision else torch.complex64, device="cuda")
        p = z2.params(lam, T, M, decomp, precision, sampling)
        res = z2.z2_run(ctx, lat.handle, p, g)
        compare_obs(res, ref, lat, lam, precision)
        assert rel_err(host(g), psi) < (1e-10 if precision else 1e-5)


def test_large_dt_quarter_turns(ctx):
    # dt = T/M beyond pi/4 takes the quarter-turn path (odd and even M)
    lat = z2.Lattice(2, (3, 3))
    ol = OLattice(2, (3, 3))
    for T, M in ((2.5, 2), (4.1, 3), (-3.3, 5)):
        psi = oracle.run(ol, 1.3, T, M, 1)
        g = torch.empty(1 << 18, dtype=torch.complex128, device="cuda")
        z2.z2_init_plus(ctx, lat.handle, z2.Z2_C128, g)
        z2.z2_evolve(ctx, lat.handle, z2.params(1.3, T, M, 1, z2.Z2_C128), g, 0, M)
        assert rel_err(host(g), psi) < 1e-11


def test_segments_equal_whole(ctx):
    lat = z2.Lattice(2, (3, 3))
    for decomp in (0, 1):
        p = z2.params(2.0, 6.0, 90, decomp, z2.Z2_C128)
        a = torch.empty(1 << 18, dtype=torch.complex128, device="cuda")
        b = torch.empty_like(a)
        z2.z2_init_plus(ctx, lat.handle, z2.Z2_C128, a)
        z2.z2_init_plus(ctx, lat.handle, z2.Z2_C128, b)
        z2.z2_evolve(ctx, lat.handle, p, a, 0, 90)
        for j0, j1 in ((0, 1), (1, 1), (1, 44), (44, 90)):
            z2.z2_evolve(ctx, lat.handle, p, b, j0, j1)
        assert rel_err(host(b), host(a)) < 1e-12


def test_3d_2x2x2_short_schedule_elementwise(ctx):
    # the 24-qubit 3D lattice at the sweep's step size, a short schedule the
    # oracle finishes in seconds; full-length runs are checked by invariants
    lat = z2.Lattice(3, (2, 2, 2))
    ol = OLattice(3, (2, 2, 2))
    lam, T, M = 3.0, 0.5, 10
    psi = oracle.run(ol, lam, T, M, 1)
    ref = oracle.observables(ol, psi, lam)
    g = torch.empty(1 << 24, dtype=torch.complex64, device="cuda")
    res = z2.z2_run(ctx, lat.handle, z2.params(lam, T, M, 1, z2.Z2_C64), g)
    compare_obs(res, ref, lat, lam, z2.Z2_C64)
    assert rel_err(host(g), psi) < 1e-5


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.0, 3.0, 4.0, 6.0])
def test_3d_config_against_oracle(ctx, lam):
    # the 3+1D configuration as stated: 2x2x2 periodic (24 links, 24
    # plaquettes, Sec. 2.1), T = 15, M = 300 symmetric steps (Eq. s), complex64,
    # every observable against the direct FP64 oracle; plus the exact
    # invariants (Gauss law, the V sector, <W> = <sigma^z> = 0, cubic symmetry)
    lat = z2.Lattice(3, (2, 2, 2))
    ol = OLattice(3, (2, 2, 2))
    T, M = 15.0, 300
    g = torch.empty(1 << 24, dtype=torch.complex64, device="cuda")
    res = z2.z2_run(ctx, lat.handle, z2.params(lam, T, M, 1, z2.Z2_C64), g)
    psi = oracle.run(ol, lam, T, M, 1)
    ref = oracle.observables(ol, psi, lam)
    d = compare_obs(res, ref, lat, lam, z2.Z2_C64)
    # the state itself: fidelity loss against the oracle's state <= 1e-6
    got = host(g)
    f = abs(np.vdot(psi, got)) ** 2 / (np.vdot(psi, psi).real * np.vdot(got, got).real)
    assert 1 - f < 1e-6, 1 - f
    assert abs(d["norm"] - 1) < 1e-5
    assert np.max(np.abs(d["star"] - 1)) < 1e-5
    assert np.max(np.abs(d["vmu"] - 1)) < 1e-5
    assert np.max(np.abs(d["wmu"])) < 1e-5
    assert np.max(np.abs(d["sigmaz"])) < 1e-5
    assert np.ptp(d["plaq"]) < 1e-5
    assert np.ptp(d["sigmax"]) < 1e-5
    assert math.isnan(d["wilson_2x2"])


def test_argument_errors(ctx):
    lat = z2.Lattice(2, (3, 3))
    g = torch.empty(1 << 18, dtype=torch.complex64, device="cuda")
    with pytest.raises(z2.Z2Error) as e:
        z2.z2_evolve(ctx, lat.handle, z2.params(1, 1, 0), g, 0, 0)
    assert e.value.code == -1 and "M" in str(e.value)
    with pytest.raises(z2.Z2Error):
        z2.z2_evolve(ctx, lat.handle, z2.params(1, 1, 10), g, 3, 11)
    with pytest.raises(z2.Z2Error):
        z2.z2_init_plus(ctx, lat.handle, z2.Z2_C64, g.data_ptr() + 8)
    with pytest.raises(z2.Z2Error):
        z2.z2_evolve(ctx, lat.handle, z2.params(float("nan"), 1, 10), g, 0, 10)
    # an empty segment is a no-op
    z2.z2_init_plus(ctx, lat.handle, z2.Z2_C64, g)
    z2.z2_evolve(ctx, lat.handle, z2.params(1, 1, 10), g, 4, 4)
    assert np.allclose(host(g), 2 ** -9)


@pytest.mark.parametrize("variant,tile_bits", [(1, 0), (2, 0), (2, 12), (1, 13), (2, 11), (1, 10), (3, 0), (3, 12), (3, 10), (3, 13), (4, 12), (4, 13), (5, 12), (5, 13)])
@pytest.mark.parametrize("d,L", [(2, (3, 3)), (2, (5, 2)), (2, (4, 3)), (3, (2, 2, 2))])
def test_kernel_variants_and_tilings(ctx, variant, tile_bits, d, L):
    # every execution variant (direct global loads / TMA pipeline) and tile
    # size gives the same evolution as the oracle
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    lam, T, M = 2.2, 1.2, 9
    psi = oracle.run(ol, lam, T, M, 1)
    z2.z2_ctx_set_option(ctx, z2.Z2_OPT_PASS_VARIANT, variant)
    z2.z2_ctx_set_option(ctx, z2.Z2_OPT_TILE_BITS, tile_bits)
    try:
        for precision in PRECS:
            g = torch.empty(1 << ol.n_links, dtype=torch.complex128 if precision else torch.complex64, device="cuda")
            z2.z2_init_plus(ctx, lat.handle, precision, g)
            z2.z2_evolve(ctx, lat.handle, z2.params(lam, T, M, 1, precision), g, 0, M)
            assert rel_err(host(g), psi) < (1e-11 if precision else 1e-5), (variant, tile_bits, precision)
            info = z2.z2_evolve_plan_info(ctx, lat.handle, z2.params(lam, T, M, 1, precision), 0, M)
            if tile_bits and tile_bits < ol.n_links and not (precision and tile_bits > 13):
                assert info.tile_bits == tile_bits
    finally:
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_PASS_VARIANT, 0)
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_TILE_BITS, 0)


@pytest.mark.parametrize("d,L", [(2, (3, 3)), (2, (4, 3)), (2, (2, 2))])
def test_autotune_then_parity(ctx, d, L):
    # the autotuner picks a tile size / kernel variant per qubit count; runs
    # afterwards use it and still agree with the oracle
    lat = z2.Lattice(d, L)
    ol = OLattice(d, L)
    g = torch.empty(1 << ol.n_links, dtype=torch.complex64, device="cuda")
    tr = z2.z2_autotune(ctx, lat.handle, z2.Z2_C64, g)
    assert tr.n_candidates >= 1 and tr.us_per_step > 0
    if ol.n_links > 14:
        assert tr.tile_bits in (12, 13, 14) and tr.variant in (1, 3, 4, 5)
    lam, T, M = 2.0, 1.0, 12
    psi = oracle.run(ol, lam, T, M, 1)
    z2.z2_init_plus(ctx, lat.handle, z2.Z2_C64, g)
    z2.z2_evolve(ctx, lat.handle, z2.params(lam, T, M), g, 0, M)
    assert rel_err(host(g), psi) < 1e-5
    if ol.n_links > 14:
        info = z2.z2_evolve_plan_info(ctx, lat.handle, z2.params(lam, T, M), 0, M)
        assert info.tile_bits == tr.tile_bits


@pytest.mark.parametrize("variant,tile_bits,low,groups", [(3, 13, 12, 3), (3, 12, 11, 4), (1, 13, 13, 3), (4, 13, 13, 3), (5, 13, 12, 3)])
def test_ring_low_group_tile(ctx, variant, tile_bits, low, groups):
    # 32 qubits (4x4): the complex64 ring runs the low group on a tile one bit
    # smaller (twice the workers) when the strided groups absorb the extra bit
    # with no extra pass; the other kernels keep one tile size
    lat = z2.Lattice(2, (4, 4))
    z2.z2_ctx_set_option(ctx, z2.Z2_OPT_PASS_VARIANT, variant)
    z2.z2_ctx_set_option(ctx, z2.Z2_OPT_TILE_BITS, tile_bits)
    try:
        info = z2.z2_evolve_plan_info(ctx, lat.handle, z2.params(3.0, 20.0, 500), 0, 500)
        assert (info.tile_bits, info.low_tile_bits, info.n_groups) == (tile_bits, low, groups)
        assert info.n_passes == 500 * (groups - 1) + 1
    finally:
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_PASS_VARIANT, 0)
        z2.z2_ctx_set_option(ctx, z2.Z2_OPT_TILE_BITS, 0)
