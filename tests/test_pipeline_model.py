"""A model of the float32 weight-gradient pipeline's barrier protocol, checked on the CPU.

Roles (as in k_wgrad_tc_f32): one producer loads chunk i into stage i mod S once the MMAs of
chunk i - S are done; T split teams take chunks i = team (mod T), each in order, and wait for
the chunk's load with an mbarrier parity wait; one MMA thread takes every chunk in order and
waits for its split. Loads complete in any order. An mbarrier parity wait for phase m passes
when the barrier's completed-phase count has the other parity, so it also passes, wrongly,
when the count is m - 1 (a load two phases old). The model explores random schedules and
checks that no wait ever passes before the phase it waits for completed: with S a multiple of
T no schedule breaks this, and with S not a multiple of T some schedule does. A second model
does the same for the convolution kernel's ring and its double-buffered TMEM accumulators."""
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


def _run_conv(S, NB, tiles, nk, seed, acc_wait=True):
    """The convolution kernel's float32-form protocol, one random schedule. Per tile nk chunks
    go round the S-stage ring (producer -> split warpgroup -> MMA thread, the MMA completion
    freeing the stage), and the tile's accumulator is one of NB TMEM buffers (MMA thread ->
    epilogue, the epilogue's arrival freeing the buffer). Returns the first wrong wait, or None.
    acc_wait=False drops the MMA thread's wait for a drained accumulator (a planted mistake)."""
    rnd = random.Random(seed)
    full, split, empty = [0] * S, [0] * S, [0] * S
    accf, acce = [0] * NB, [0] * NB
    nch = tiles * nk
    issued, inflight, split_next = 0, [], 0
    mma_it, mma_tile, mma_pending, acc_busy = 0, 0, [], set()
    epi_tile, epi_pending = 0, []

    def passes(count, phase):
        return (count & 1) != (phase & 1)

    while epi_tile < tiles or epi_pending:
        acts = []
        if issued < nch and (issued < S or passes(empty[issued % S], issued // S - 1)):
            acts.append(("issue",))
        acts += [("land", c) for c in inflight]
        if split_next < nch and passes(full[split_next % S], split_next // S):
            acts.append(("split",))
        if mma_tile < tiles:
            buf, lt = mma_tile % NB, mma_tile
            if acc_wait and mma_it % nk == 0 and lt >= NB and not passes(acce[buf], lt // NB - 1):
                pass  # the accumulator is still being drained
            elif passes(split[mma_it % S], mma_it // S):
                acts.append(("mma",))
        acts += [("mmadone", c) for c in mma_pending]
        if epi_tile < tiles and passes(accf[epi_tile % NB], epi_tile // NB):
            acts.append(("epi",))
        acts += [("epidone", t) for t in epi_pending]
        if not acts:
            return ("deadlock", seed)
        a = rnd.choice(acts)
        if a[0] == "issue":
            if issued >= S and empty[issued % S] < issued // S:
                return ("overwrite", issued, seed)
            inflight.append(issued)
            issued += 1
        elif a[0] == "land":
            inflight.remove(a[1])
            full[a[1] % S] += 1
        elif a[0] == "split":
            i = split_next
            if full[i % S] < i // S + 1:
                return ("stale load", i, seed)
            split[i % S] += 1
            split_next += 1
        elif a[0] == "mma":
            i, t = mma_it, mma_tile
            if split[i % S] < i // S + 1:
                return ("stale split", i, seed)
            if i % nk == 0:
                if t % NB in acc_busy:
                    return ("accumulator overwritten", t, seed)
                acc_busy.add(t % NB)
            last = (i + 1) % nk == 0
            mma_pending.append((i, t if last else -1))
            mma_it += 1
            if last:
                mma_tile += 1
        elif a[0] == "mmadone":
            mma_pending.remove(a[1])
            i, t = a[1]
            empty[i % S] += 1
            if t >= 0:
                accf[t % NB] += 1
        elif a[0] == "epi":
            t = epi_tile
            if accf[t % NB] < t // NB + 1:
                return ("stale accumulator", t, seed)
            epi_pending.append(t)
            epi_tile += 1
        else:
            epi_pending.remove(a[1])
            acc_busy.discard(a[1] % NB)
            acce[a[1] % NB] += 1
    return None


@pytest.mark.parametrize("S,NB,nk", [(2, 2, 1), (2, 1, 3), (3, 2, 4), (4, 2, 2), (4, 1, 16)])
def test_conv_pipeline_waits_pass_only_on_their_phase(S, NB, nk):
    for seed in range(300):
        assert _run_conv(S, NB, 7, nk, seed) is None


def test_conv_model_catches_a_missing_accumulator_wait():
    bad = [r for r in (_run_conv(2, 2, 7, 2, seed, acc_wait=False) for seed in range(300)) if r]
    assert bad and all(r[0] == "accumulator overwritten" for r in bad)
