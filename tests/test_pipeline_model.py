"""A model of the float32 weight-gradient pipeline's barrier protocol, checked on the CPU.

Roles (as in k_wgrad_tc_f32): one producer loads chunk i into stage i mod S once the MMAs of
chunk i - S are done; T split teams take chunks i = team (mod T), each in order, and wait for
the chunk's load with an mbarrier parity wait; one MMA thread takes every chunk in order and
waits for its split. Loads complete in any order. An mbarrier parity wait for phase m passes
when the barrier's completed-phase count has the other parity, so it also passes, wrongly,
when the count is m - 1 (a load two phases old). The model explores random schedules and
checks that no wait ever passes before the phase it waits for completed: with S a multiple of
T no schedule breaks this, and with S not a multiple of T some schedule does."""
import random

import pytest


def _run(S, T, nk, seed):
    """One random schedule; returns the first wrong wait found, or None."""
    rnd = random.Random(seed)
    full = [0] * S    # completed phases of each stage's load barrier
    split = [0] * S   # completed phases of each stage's split barrier
    empty = [0] * S   # completed phases of each stage's MMA-done barrier
    issued = 0        # next chunk the producer loads
    inflight = []     # loads issued, not yet landed (chunk numbers)
    team_next = list(range(T))  # next chunk of each team
    mma_next = 0
    mma_inflight = []  # chunks whose MMAs are issued, not done

    def passes(count, i):  # the parity wait of chunk i on a barrier with `count` completions
        return (count & 1) != ((i // S) & 1)

    while mma_next < nk or mma_inflight:
        acts = []
        if issued < nk and (issued < S or empty[issued % S] >= issued // S):
            acts.append(("issue",))
        for c in inflight:
            acts.append(("land", c))
        for t in range(T):
            i = team_next[t]
            if i < nk and passes(full[i % S], i):
                acts.append(("split", t))
        if mma_next < nk and passes(split[mma_next % S], mma_next):
            acts.append(("mma",))
        for c in mma_inflight:
            acts.append(("mmadone", c))
        if not acts:
            return ("deadlock", seed)
        a = rnd.choice(acts)
        if a[0] == "issue":
            inflight.append(issued)
            issued += 1
        elif a[0] == "land":
            inflight.remove(a[1])
            full[a[1] % S] += 1
        elif a[0] == "split":
            i = team_next[a[1]]
            if full[i % S] < i // S + 1:  # the wait passed on an older phase
                return ("stale load", i, seed)
            split[i % S] += 1
            team_next[a[1]] += T
        elif a[0] == "mma":
            i = mma_next
            if split[i % S] < i // S + 1:
                return ("stale split", i, seed)
            mma_inflight.append(i)
            mma_next += 1
        else:
            mma_inflight.remove(a[1])
            empty[a[1] % S] += 1
    return None


@pytest.mark.parametrize("S,T", [(6, 2), (6, 3), (6, 1), (4, 4), (4, 2), (2, 2), (5, 1)])
def test_stage_count_multiple_of_teams_is_safe(S, T):
    for seed in range(300):
        assert _run(S, T, 40, seed) is None


@pytest.mark.parametrize("S,T", [(6, 4), (5, 2), (3, 2)])
def test_other_stage_counts_can_split_a_stale_load(S, T):
    bad = [r for r in (_run(S, T, 40, seed) for seed in range(2000)) if r is not None]
    assert bad and all(r[0] == "stale load" for r in bad)
