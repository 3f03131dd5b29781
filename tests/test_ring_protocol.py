"""A model of the buffer protocol of the complex64 TMA ring pass kernel
(pass_kernel_ring in paper_1910_08020_gb300/csrc/pass_packed.cuh), checked on
the CPU with an event simulation.

One CTA runs NW workers over NB > NW shared-memory buffers.  Local tile n lives
in buffer n % NB and is transformed by worker n % NW; after storing tile n, its
worker refills the buffer with tile n + NB.  Each buffer has one mbarrier whose
phase completes when a load lands, and a waiter tests a phase by its parity.

When NB is not a multiple of NW, consecutive loads into one buffer are
consumed by different workers.  A worker that tests the parity of load u while load u - 1 is still in flight sees
the barrier in phase u - 1, whose parity differs from u's, so the test reports
the finished phase u - 2 and the worker reads a buffer that is still being
written.  The kernel therefore waits first until the buffer's previous load has
been observed (a per-buffer counter in shared memory).  The model checks that
with that gate no worker ever reads a buffer before its load landed and no
buffer ever gets two loads in flight, for every (NW, NB) the kernel
instantiates, and that without the gate slow loads do break it.
"""
import heapq
import random

import pytest

# (workers, buffers) of RingTile for tile bits 13, 12, 11, 10 with 16 pairs per
# thread and for tile bits 13, 12 with 32 pairs per thread
CONFIGS = [(2, 3), (4, 6), (8, 12), (8, 16)]


class Broken(Exception):
    pass


def simulate(nw, nb, n_tiles, gated, seed, load_max):
    rnd = random.Random(seed)
    phases = [0] * nb      # completed phases of each buffer's barrier
    landed = [None] * nb   # tile whose data is complete in the buffer
    inflight = [None] * nb
    seen = [0] * nb        # loads of each buffer a worker has observed
    events = []

    def load(k, n, now):
        if inflight[k] is not None:
            raise Broken(f"buffer {k}: load of tile {n} while tile {inflight[k]} is in flight")
        inflight[k] = n
        heapq.heappush(events, (now + rnd.uniform(0.05, load_max), 0, "land", (k, n)))

    for n in range(min(nb, n_tiles)):
        load(n, n, 0.0)
    next_tile = list(range(nw))
    for w in range(nw):
        heapq.heappush(events, (0.0, 1, "poll", w))
    done = 0
    while events:
        t, _, kind, data = heapq.heappop(events)
        if kind == "land":
            k, n = data
            inflight[k], landed[k] = None, n
            phases[k] += 1
        elif kind == "poll":
            w = data
            n = next_tile[w]
            if n >= n_tiles:
                continue
            k, use = n % nb, n // nb
            ready = (not gated or seen[k] == use) and (phases[k] & 1) != (use & 1)
            if not ready:
                heapq.heappush(events, (t + 0.01, 1, "poll", w))
                continue
            if landed[k] != n:
                raise Broken(f"worker {w} read buffer {k} for tile {n} before its load landed")
            seen[k] = use + 1
            heapq.heappush(events, (t + rnd.uniform(0.5, 1.5), 1, "done", (w, n)))
        else:
            w, n = data
            k = n % nb
            landed[k] = None
            if n + nb < n_tiles:
                load(k, n + nb, t)
            next_tile[w] = n + nw
            done += 1
            heapq.heappush(events, (t, 1, "poll", w))
    assert done == n_tiles


@pytest.mark.parametrize("nw,nb", CONFIGS)
def test_gated_wait_never_reads_early(nw, nb):
    # loads up to five tiles of compute long: far slower than any real copy
    for seed in range(60):
        for load_max in (0.3, 2.0, 5.0):
            simulate(nw, nb, 300, True, seed, load_max)


@pytest.mark.parametrize("nw,nb", [c for c in CONFIGS if c[1] % c[0]])
def test_parity_alone_breaks_with_slow_loads(nw, nb):
    # the ungated wait is exact while loads are shorter than the compute...
    for seed in range(20):
        simulate(nw, nb, 300, False, seed, 0.3)
    # ...and reads early once a load outlives two tiles of the other workers
    broken = 0
    for seed in range(60):
        try:
            simulate(nw, nb, 300, False, seed, 5.0)
        except Broken:
            broken += 1
    assert broken > 0


@pytest.mark.parametrize("nw,nb", [c for c in CONFIGS if c[1] % c[0] == 0])
def test_parity_alone_is_exact_when_buffers_belong_to_one_worker(nw, nb):
    # with NB a multiple of NW every load of a buffer goes to the same worker,
    # which observes them in order, so the parity test alone cannot alias
    for seed in range(60):
        simulate(nw, nb, 300, False, seed, 5.0)
