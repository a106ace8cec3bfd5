"""Index arithmetic of the decoupled fit's feature ring, checked on the host.

The streamed-feature ring of k_fit_x (xpipe_issue, xpass_pipe and xpipe_drain
in csrc/mdhp_fitx.cuh) runs an endless cyclic sequence of bulk-copy fills
over a window's stages: fill g holds stage (g - base) mod nst, lands in
buffer g mod D, and its consumer waits on that buffer's mbarrier for the
(g // D)-th completion (phase parity (g // D) & 1).  This test replays those
formulas step by step: the window start (D fills issued), every evaluation
(a stage per fill, the next fill issued after each consumed one), the drain
after the last evaluation, and a wait that gives up at any stage of any
evaluation (the fill it waited for stays owed and the drain waits from it
on).  It checks the invariants the kernel relies on:

* a consumer reads the stage it expects, from a fill that was issued;
* a parity wait cannot be satisfied by a different completion: the next
  fill into a buffer is issued only after the previous one was consumed, so
  at most one completion per buffer is outstanding;
* the drain waits exactly for the fills issued and not consumed, so no copy
  is still writing into the ring when the CTA moves on."""
import itertools

import pytest


class Ring:
    """The kernel's counters (used, issued, base) and the per-buffer history."""

    def __init__(self, D):
        self.D = D
        self.used = 0
        self.issued = 0
        self.base = 0
        self.nst = 1
        self.fills = {}        # fill index -> stage it carries
        self.consumed = set()
        self.completions = [0] * D  # fills that have landed per buffer

    # xpipe_issue: g = issued++; stage (g - base) mod nst into buffer g mod D
    def issue(self):
        g = self.issued
        self.issued += 1
        slot = g % self.D
        if g >= self.D:  # the buffer's previous fill must have been consumed
            assert (g - self.D) in self.consumed, ("buffer reused before consumed", g)
        self.fills[g] = (g - self.base) % self.nst
        self.completions[slot] += 1  # the copy lands (completion of the slot's barrier)
        return g

    # the wait of fill g: parity (g // D) & 1 on buffer g mod D
    def wait(self, g):
        slot = g % self.D
        assert g in self.fills, ("waiting for a fill never issued", g)
        # the completion the waiter expects is the (g // D)-th of its buffer;
        # with at most one completion outstanding, parity identifies it
        expected = g // self.D + 1
        assert self.completions[slot] == expected, (g, self.completions[slot], expected)

    def start_window(self, nst):
        self.nst = nst
        self.base = self.used
        self.issued = self.used
        for _ in range(self.D):
            self.issue()

    # one evaluation (xpass_pipe); gives up at stage fail_at (None: never)
    def evaluate(self, fail_at=None):
        for s in range(self.nst):
            g = self.used
            if fail_at == s:
                return False  # the wait gave up: fill g is still owed
            self.wait(g)
            assert self.fills[g] == s, ("stage mismatch", g, self.fills[g], s)
            self.consumed.add(g)
            self.used += 1
            self.issue()
        return True

    # xpipe_drain: waits used .. used + D - 1 (each with the full bound)
    def drain(self):
        outstanding = set(range(self.used, self.issued))
        waited = set()
        for _ in range(self.D):
            g = self.used
            self.used += 1
            self.wait(g)
            self.consumed.add(g)
            waited.add(g)
        assert waited == outstanding, ("drain does not match the fills in flight", waited, outstanding)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 8])
def test_windows_of_every_length_stay_in_step(D):
    r = Ring(D)
    for nst, iters in itertools.product([1, 2, 3, 5, 8, 13], [1, 2, 3, 7]):
        r.start_window(nst)
        for _ in range(iters):
            assert r.evaluate()
        r.drain()
        assert r.issued == r.used


@pytest.mark.parametrize("D", [1, 2, 3, 4])
def test_timeout_at_any_stage_is_drained_exactly(D):
    for nst in (1, 2, 3, 6):
        for k_fail in range(3):
            for s_fail in range(nst):
                r = Ring(D)
                # an earlier window, then the window whose wait gives up
                r.start_window(3)
                assert r.evaluate()
                r.drain()
                r.start_window(nst)
                for k in range(k_fail + 1):
                    ok = r.evaluate(fail_at=s_fail if k == k_fail else None)
                    if not ok:
                        break
                assert not ok
                r.drain()  # waits from the owed fill on
                assert r.issued == r.used
                # the ring is consistent again for the next window
                r.start_window(nst)
                assert r.evaluate()
                r.drain()
