"""CPU check of the stage schedule of the bulk-copy row kernel
(k_step_row_copy, csrc/step_kernels.cuh): velocity i is copied into stage
i % NST and waited for with parity (i // NST) % 2; the first warp issues
velocities 0 .. NST-1 before the loop and, after the block barrier of group
g (velocities 3g .. 3g+2), the velocities up to 3g + 3 + NST.  The model
replays that order for the velocity counts of the built sets and checks the
invariants the kernel's correctness rests on:
  * a velocity is issued before any thread waits for it;
  * when a thread waits for velocity i, its stage holds velocity i's phase
    and no later one (the parity test cannot tell phase k from k + 2);
  * a stage is never refilled while a thread may still read it (reads of a
    group happen before its barrier, refills after it), including the reads
    of the unused slots of a last, partial group;
  * at exit every issued velocity has been waited for (no copy lands after
    the block is gone).
"""
import pytest

GV = 3


def _replay(Q, NST):
    stage_of = {}            # stage -> list of velocities issued into it, in order
    issued = []
    in_flight = set()        # velocities issued, not yet waited for

    def issue(i):
        s = i % NST
        stage_of.setdefault(s, []).append(i)
        issued.append(i)
        in_flight.add(i)

    for i in range(min(NST, Q)):
        issue(i)
    n_issued = min(NST, Q)
    for i0 in range(0, Q, GV):
        # waits of the group
        for u in range(GV):
            i = i0 + u
            if i >= Q:
                continue
            s = i % NST
            assert i in issued, f"velocity {i} waited before it was issued"
            hist = stage_of[s]
            k = hist.index(i)
            assert k == i // NST, "stage holds another phase"
            assert hist[-1] == i, f"stage {s} already refilled past velocity {i}"
            assert (k & 1) == ((i // NST) & 1)
            in_flight.discard(i)
        # reads of the group's stages (the slots past Q read a stale stage)
        for u in range(GV):
            s = (i0 + u) % NST
            live = [j for j in stage_of.get(s, []) if j in in_flight]
            assert not live, f"stage {s} read while velocity {live} is in flight"
        # barrier, then refill
        end = min(i0 + GV + NST, Q)
        for j in range(n_issued, end):
            issue(j)
        n_issued = max(n_issued, end)
    assert not in_flight, f"copies still in flight at exit: {sorted(in_flight)}"
    assert sorted(issued) == list(range(Q))


@pytest.mark.parametrize("Q", [19, 45])
def test_stage_schedule_of_the_bulk_copy_row_kernel(Q):
    _replay(Q, 6)


@pytest.mark.parametrize("NST", [3, 4, 9])
def test_schedule_holds_for_other_stage_counts(NST):
    """Refills after the barrier only target stages of already-read
    velocities, so any stage count of at least one group works (the kernel
    uses 6: two groups of look-ahead)."""
    _replay(45, NST)


def test_schedule_model_detects_too_few_stages():
    """With fewer stages than a group, a thread would wait for a velocity
    that no copy was issued for yet: the model fails."""
    with pytest.raises(AssertionError):
        _replay(45, 2)
