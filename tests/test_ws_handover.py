"""The hand-over protocol of the warp-specialised small-neighbourhood LP
(k_lp_small32_ws), modelled on the CPU.

The kernel's two roles exchange batches through kWsSlots = 3 shared-memory
buffers; buffer s has a named barrier FULL_s (the pivot warps arrive after
writing a batch into it, the FP64 warps wait there before reading) and
EMPTY_s (the FP64 warps arrive after reading, the pivot warps wait there
before writing the buffer again).  A named barrier completes a generation
when every thread of the block has arrived or waited on it; an arrival that
no wait of the other role matches would leave a generation part-filled.

The model replays the two roles' sequences of barrier operations, as the
kernel's loops issue them, under random interleavings and checks that the
block never deadlocks, that no role reaches a barrier twice within one
generation, that a batch is read only after it was written into its buffer,
that a buffer is overwritten only after its batch was read, and that no
barrier is left part-filled when both loops end.  It also checks that the
protocol fails these checks when the last EMPTY arrivals are not left out,
or with a buffer too few for the waits.
"""
import random

import pytest

SLOTS = 3


def programs(rounds, slots=SLOTS, skip_last_empty=True):
    """The barrier operations of the pivot role (P) and the FP64 role (F) of
    one block that takes `rounds` batches, in the kernel's loop order."""
    piv = []
    for r in range(rounds):
        s = r % slots
        if r >= slots:
            piv.append(("sync", "E%d" % s))
        piv.append(("write", r))
        piv.append(("arrive", "F%d" % s))
    fin = []
    for d in range(rounds):
        s = d % slots
        fin.append(("sync", "F%d" % s))
        fin.append(("read", d))
        if not skip_last_empty or d + slots < rounds:
            fin.append(("arrive", "E%d" % s))
    return {"P": piv, "F": fin}


def run(prog, rng, slots=SLOTS):
    """One random interleaving; raises AssertionError on any violation."""
    pc = {"P": 0, "F": 0}
    arrived = {}   # barrier -> roles arrived in its current generation
    gen = {}       # barrier -> completed generations
    waiting = {}   # role -> (barrier, generation it waits for)
    written, read, held = set(), set(), {}
    while True:
        runnable = []
        for role in ("P", "F"):
            if pc[role] >= len(prog[role]):
                continue
            if role in waiting:
                bar, g = waiting[role]
                if gen.get(bar, 0) > g:
                    runnable.append(role)
            else:
                runnable.append(role)
        if not runnable:
            assert all(pc[r] >= len(prog[r]) for r in pc), "deadlock"
            assert all(not v for v in arrived.values()), "barrier left part-filled"
            return
        role = rng.choice(runnable)
        if role in waiting:
            del waiting[role]
            pc[role] += 1
            continue
        op, arg = prog[role][pc[role]]
        if op in ("arrive", "sync"):
            now = arrived.setdefault(arg, set())
            assert role not in now, "a role reached a barrier twice in one generation"
            now.add(role)
            g = gen.get(arg, 0)
            if len(now) == 2:
                arrived[arg] = set()
                gen[arg] = g + 1
            if op == "sync":
                waiting[role] = (arg, g)
                continue
            pc[role] += 1
        elif op == "write":
            s = arg % slots
            if s in held:
                assert held[s] in read, "buffer overwritten before its batch was read"
            held[s] = arg
            written.add(arg)
            pc[role] += 1
        else:
            assert arg in written and held[arg % slots] == arg, "batch read before it was written"
            read.add(arg)
            pc[role] += 1


def test_handover_protocol_holds_for_every_round_count():
    rng = random.Random(1508)
    for rounds in range(0, 30):
        prog = programs(rounds)
        for _ in range(60):
            run(prog, rng)


def test_handover_checks_catch_a_broken_protocol():
    rng = random.Random(7)
    # every EMPTY arrival kept: the last ones are never waited for
    with pytest.raises(AssertionError, match="part-filled"):
        for _ in range(20):
            run(programs(5, skip_last_empty=False), rng)
    # the pivot role waiting on EMPTY one round too late for two buffers'
    # worth of batches ahead: the model with 2 buffers but the waits of 3
    prog = programs(6, slots=3)
    with pytest.raises(AssertionError):
        for _ in range(200):
            run(prog, rng, slots=2)
