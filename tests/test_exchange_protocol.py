"""A model of the tridiagonalisation's cross-block exchange (no GPU), following k_tridiag: column j
is owned by block j mod G; during step k the owners of the columns j >= k + 2 publish the words of
step k + 1 (entry t = j - k - 2) tagged with the epoch (k + 1) mod 4 into buffer (k + 1) mod 2;
at step k every running block waits until all the words it reads (entries t < N - k - 1 of buffer
k mod 2) carry the epoch k mod 4.  The buffers start with every word at epoch 3 (the 0x03 byte
fill).  A block leaves once it owns no column >= k + 2, except the block owning the last column,
which writes the outputs; so every block still reading step k publishes words of step k + 1.
Random interleavings of the blocks' single-word reads and writes check that a block never accepts
a word of another step and that the exchange always completes.  Without the early exit, a block
whose columns are all done could fall behind and meet the words of step k + 2 (or, 4 steps behind,
accept those of step k + 4): the model then fails, which is why the kernel has the exit."""
import random

import pytest


def simulate(N, G, seed, early_exit=True):
    rng = random.Random(seed)
    buf = [[(-1, 3)] * N for _ in range(2)]          # (true step, epoch) of each word
    owned = [[j for j in range(N) if j % G == b] for b in range(G)]
    ob = (N - 1) % G                                  # the block owning the last column
    # per block: a queue of actions; ('w', step, t) writes P_step[t]; ('r', step) reads all of P_step
    def program(b):
        acts = [("w", 0, j - 1) for j in owned[b] if j >= 1]               # prologue: step 0
        for k in range(N - 2):
            if early_exit and b != ob and max(owned[b]) < k + 2:
                break
            acts.append(("r", k))
            if k + 3 < N:                                                  # step k+1 exists
                acts += [("w", k + 1, j - (k + 2)) for j in owned[b] if j >= k + 2]
        return acts
    progs = [program(b) for b in range(G)]
    pos = [0] * G
    steps = 0
    while any(pos[b] < len(progs[b]) for b in range(G)):
        b = rng.choice([x for x in range(G) if pos[x] < len(progs[x])])
        act = progs[b][pos[b]]
        if act[0] == "w":
            _, k, t = act
            buf[k & 1][t] = (k, k & 3)
            pos[b] += 1
        else:
            k = act[1]
            words = buf[k & 1][:N - k - 1]
            if all(e == (k & 3) for _, e in words):                        # every word carries the epoch
                assert all(s == k for s, _ in words), (b, k, words)         # ... and belongs to step k
                pos[b] += 1
        steps += 1
        assert steps < 2_000_000, "exchange did not complete"
    return steps


@pytest.mark.parametrize("N,G", [(3, 1), (8, 2), (17, 4), (40, 9), (96, 12)])
def test_exchange_never_accepts_a_stale_word(N, G):
    for seed in range(20):
        simulate(N, G, seed)


def test_without_the_early_exit_a_finished_block_can_fall_behind():
    failed = 0
    for seed in range(20):
        try:
            simulate(17, 4, seed, early_exit=False)
        except AssertionError:
            failed += 1
    assert failed > 0
