"""Host-side logic of the serving loop (no GPU): the range allocator that
backs admission by free device memory."""
from __future__ import annotations

import numpy as np

from paper_1411_5283_gb300.serve import RangeAllocator, Request


def test_allocator_first_fit_and_coalesce():
    a = RangeAllocator(100, align=1)
    x = a.alloc(30)
    y = a.alloc(30)
    z = a.alloc(30)
    assert (x, y, z) == (0, 30, 60)
    assert a.alloc(20) == -1          # only 10 left
    a.release(y, 30)
    assert a.alloc(25) == 30          # first fit into the hole
    a.release(30, 25)
    a.release(x, 30)
    a.release(z, 30)
    assert a.free == [(0, 100)]       # fully coalesced
    assert a.free_total == 100


def test_allocator_alignment():
    a = RangeAllocator(64, align=16)
    assert a.alloc(1) == 0 and a.alloc(17) == 16 and a.alloc(16) == 48
    assert a.alloc(1) == -1


def test_allocator_random_no_overlap():
    rng = np.random.default_rng(0)
    a = RangeAllocator(10_000, align=4)
    live = {}
    for step in range(3000):
        if live and rng.random() < 0.45:
            k = list(live)[rng.integers(len(live))]
            a.release(k, live.pop(k))
        else:
            n = int(rng.integers(1, 400))
            s = a.alloc(n)
            if s >= 0:
                n4 = (n + 3) // 4 * 4
                for t, m in live.items():
                    m4 = (m + 3) // 4 * 4
                    assert s + n4 <= t or t + m4 <= s
                live[s] = n
    for k, n in list(live.items()):
        a.release(k, n)
    assert a.free == [(0, 10_000)]


def test_request_slots():
    r = Request(0, rec=np.zeros((7, 8), np.uint8), ln=np.ones(7, np.uint8))
    assert r.n_slots == 7 and not r.is_text
    t = Request(1, text=b"abc def")
    assert t.is_text and t.n_slots == len(b"abc def") // 2 + 1


def _rec_request(rid, n):
    return Request(rid, rec=np.zeros((n, 8), np.uint8), ln=np.ones(n, np.uint8))


def test_admission_fifo_and_oversize():
    from paper_1411_5283_gb300.serve import Admission
    adm = Admission(n_slots=256, text_bytes=64, max_list_words=200)
    big = _rec_request(0, 300)
    adm.submit(big, 0.0)
    assert adm.rejected == [big] and big.status == 7       # more than the arena
    too_long = _rec_request(1, 250)
    adm.submit(too_long, 0.0)
    assert too_long in adm.rejected                          # above the per-list limit
    a, b, c = _rec_request(2, 100), _rec_request(3, 120), _rec_request(4, 20)
    for r in (a, b, c):
        adm.submit(r, 0.0)
    adm.admit(1.0)
    assert adm.admitted == [a, b] and list(adm.waiting) == [c]  # c waits behind the head
    adm.admitted.clear()          # a and b "launched"
    adm.release(a)
    adm.admit(2.0)
    assert adm.admitted == [c]


def test_kept_results_never_block_the_queue_forever():
    """With results kept (nothing released), a request that no longer fits is
    rejected once nothing is admitted or in flight, instead of waiting for
    memory that nothing will free; the requests behind it still run."""
    from paper_1411_5283_gb300.serve import Admission
    adm = Admission(n_slots=256, text_bytes=64, max_list_words=256)
    first, second, third = _rec_request(0, 200), _rec_request(1, 200), _rec_request(2, 32)
    for r in (first, second, third):
        adm.submit(r, 0.0)
    adm.admit(0.0)
    assert adm.admitted == [first]
    adm.admitted.clear()          # launched and completed; its slots are kept
    adm.admit(1.0)
    assert adm.admitted == [] and list(adm.waiting) == [second, third]
    adm.unblock(in_flight=True, now=1.0)    # something may still free memory: wait
    assert list(adm.waiting) == [second, third]
    adm.unblock(in_flight=False, now=2.0)   # nothing will: reject the head, go on
    assert adm.rejected == [second] and second.status == 7
    assert adm.admitted == [third] and not adm.waiting
