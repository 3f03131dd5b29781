"""The allocation-free reduction z2_zsums_static, for callers that cannot
allocate device memory: it needs no context and keeps its scratch in a fixed
array inside the library.  Two calls in a row must each agree with z2_zsums
(which uses context-owned scratch) and with the FP64 oracle within the
tolerance of the other reduction tests, at sizes that use every block count
of the call (1 block at 8 qubits up to the full 1024); a smaller call after a
full-size one must not see the larger call's leftover partial sums; an
oversized request is refused with a message.  This file is collected last,
so a run that stops at the first failure has already run every other test."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_1910_08020_gb300 as z2
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


def masks_for(n, seed, count):
    rng = np.random.default_rng(seed)
    return np.concatenate([[0], rng.integers(0, 1 << n, size=count - 1, dtype=np.uint64)]).astype(np.uint64)


def check(ctx, n, precision, psi, m, tol):
    got = z2.z2_zsums_static(n, precision, psi, m)
    want = z2.z2_zsums(ctx, n, precision, psi, m)
    assert np.max(np.abs(got - want)) < tol, np.max(np.abs(got - want))
    torch.cuda.synchronize()
    ref = oracle.zsums(psi.cpu().numpy().astype(np.complex128), m)  # the device copy, in FP64
    assert np.max(np.abs(got - ref)) < tol, np.max(np.abs(got - ref))
    assert abs(got[0] - 1.0) < 1e-5  # mask 0 is the norm
    return got


@pytest.mark.parametrize("n,precision", [(8, z2.Z2_C64), (12, z2.Z2_C64), (14, z2.Z2_C128), (18, z2.Z2_C64),
                                         (24, z2.Z2_C64), (28, z2.Z2_C64), (18, z2.Z2_C128)])
def test_static_scratch_matches_context_scratch(ctx, n, precision):
    dt = torch.complex128 if precision == z2.Z2_C128 else torch.complex64
    psi = torch.from_numpy(workloads.random_state(n, seed=n)).to(dt).cuda()
    tol = 1e-12 if precision == z2.Z2_C128 else 1e-6
    for seed, count in ((1, 32), (2, 17)):  # two calls in a row share the array
        check(ctx, n, precision, psi, masks_for(n, seed + n, count), tol)


def test_static_scratch_smaller_after_larger(ctx):
    # 1024 blocks (18 qubits) fill every partial slot; a 10-qubit call then
    # uses 4 blocks and must add only its own
    big = torch.from_numpy(workloads.random_state(18, seed=5)).to(torch.complex64).cuda()
    check(ctx, 18, z2.Z2_C64, big, masks_for(18, 7, 32), 1e-6)
    small = torch.from_numpy(workloads.random_state(10, seed=6)).to(torch.complex64).cuda()
    check(ctx, 10, z2.Z2_C64, small, masks_for(10, 8, 32), 1e-6)


def test_static_scratch_limits(ctx):
    psi = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    with pytest.raises(z2.Z2Error) as e:
        z2.z2_zsums_static(10, z2.Z2_C64, psi, np.arange(33, dtype=np.uint64))
    assert "32" in str(e.value)
