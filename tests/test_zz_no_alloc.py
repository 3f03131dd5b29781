"""The allocation-free reduction z2_zsums_static, for callers that cannot
allocate device memory: it needs no context and keeps its scratch in a fixed
array inside the library.  Two calls in a row must each agree with z2_zsums
(which uses context-owned scratch) within the tolerance of the other
reduction tests; an oversized request is refused with a message.  This file
is collected last, so a run that stops at the first failure has already run
every other test."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("n,precision", [(18, z2.Z2_C64), (24, z2.Z2_C64), (28, z2.Z2_C64), (18, z2.Z2_C128)])
def test_static_scratch_matches_context_scratch(ctx, n, precision):
    dt = torch.complex128 if precision == z2.Z2_C128 else torch.complex64
    psi = torch.from_numpy(workloads.random_state(n, seed=n)).to(dt).cuda()
    tol = 1e-12 if precision == z2.Z2_C128 else 1e-6
    for call, (seed, count) in enumerate(((1, 32), (2, 17))):  # two calls in a row share the array
        m = masks_for(n, seed + n, count)
        got = z2.z2_zsums_static(n, precision, psi, m)
        want = z2.z2_zsums(ctx, n, precision, psi, m)
        assert np.max(np.abs(got - want)) < tol, (call, np.max(np.abs(got - want)))
        assert abs(got[0] - 1.0) < 1e-5  # mask 0 is the norm


def test_static_scratch_limits():
    psi = torch.zeros(1 << 10, dtype=torch.complex64, device="cuda")
    with pytest.raises(z2.Z2Error) as e:
        z2.z2_zsums_static(10, z2.Z2_C64, psi, np.arange(33, dtype=np.uint64))
    assert "32" in str(e.value)
