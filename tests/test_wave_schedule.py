"""Host-side model of the wavefront solve's scheduling (few-system triangular
solves, Sec. 3.2 with the evaluated factor of Sec. 3.3): CTAs take tickets in
the order they start, ticket tk is row step tk // S of system tk % S, a row
waits for the solved blocks before it (forward) or after it (backward) in the
order they are solved, and a CTA holds its SM until it has published its own
block.

The model replays that arithmetic with CTAs started in random order under any
number of resident CTAs (1 up to all), and checks that every CTA finishes (no
wait depends on a CTA that has not started), that every block is published
exactly once, and that every index into the exchange buffer and the solution
stays inside the sizes the workspace plan gives them.  It also replays the
wait check (tickets numbered from S, the first row step left out): there every
CTA's first wait is on block 0, which nothing publishes."""
import random

import pytest

TB = 64


def ticket_to_row(tk, S, nt, direction):
    step, sidx = divmod(tk, S)
    return sidx, (step if direction == 0 else nt - 1 - step)


def waits_of(I, nt, direction):
    """The blocks row I applies, in the order the kernel waits for them."""
    return list(range(I)) if direction == 0 else list(range(nt - 1, I, -1))


def run_schedule(S, nt, resident, direction, seed, tk0=0, ncta=None):
    """Returns (finished CTAs, published blocks, rows left waiting)."""
    rng = random.Random(seed)
    ncta = S * nt - tk0 if ncta is None else ncta
    ticket = tk0
    pending = ncta                      # CTAs not yet started
    running = []                        # [sidx, I, position in its wait list]
    published = set()
    finished = 0
    while pending or running:
        # the hardware may start any waiting CTA when a slot is free; which one
        # does not matter for the ticket, which is taken at start
        while pending and len(running) < resident:
            sidx, I = ticket_to_row(ticket, S, nt, direction)
            ticket += 1
            pending -= 1
            running.append([sidx, I, 0])
        progressed = False
        rng.shuffle(running)
        for cta in list(running):
            sidx, I, pos = cta
            need = waits_of(I, nt, direction)
            while pos < len(need) and (sidx, need[pos]) in published:
                pos += 1
                progressed = True
            cta[2] = pos
            if pos == len(need):
                assert (sidx, I) not in published
                published.add((sidx, I))
                running.remove(cta)
                finished += 1
                progressed = True
        if not progressed and not pending:
            return finished, published, running
        if not progressed and len(running) == resident:
            return finished, published, running
    return finished, published, running


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("S,nt", [(1, 1), (1, 5), (5, 16), (5, 32), (15, 32), (30, 7), (152, 4)])
def test_every_cta_finishes_under_any_residency(S, nt, direction):
    total = S * nt
    for resident in sorted({1, 2, 3, S, max(1, total // 3), total}):
        for seed in range(3):
            finished, published, stuck = run_schedule(S, nt, resident, direction, seed)
            assert not stuck and finished == total, (S, nt, resident, seed)
            assert published == {(s, i) for s in range(S) for i in range(nt)}


def test_a_wait_is_only_on_smaller_tickets():
    for S, nt in [(3, 9), (5, 32), (152, 2)]:
        for direction in (0, 1):
            for tk in range(S * nt):
                sidx, I = ticket_to_row(tk, S, nt, direction)
                for J in waits_of(I, nt, direction):
                    step_j = J if direction == 0 else nt - 1 - J
                    assert step_j * S + sidx < tk


@pytest.mark.parametrize("c", [1, 4, 5, 10, 12, 13, 32])
@pytest.mark.parametrize("k,tcount,nt,q", [(5, 1, 32, 1), (5, 3, 16, 101), (2, 1, 2, 1)])
def test_buffer_indices_stay_in_bounds(c, k, tcount, nt, q):
    """Indices the kernel forms: exchange values xs + J*64*c + e (polled) and
    xs + row*c + o (published), xs = sidx*dp*c inside a pass of S*dp*c values;
    the polled groups 4*(tid + 256*u) of a block; and the shared-memory slot
    k*ZR + (o & 3)*NJP + (o >> 2) of the staged block."""
    S, dp = k * tcount, nt * TB
    nvals = S * dp * c
    nj = 1 if c <= 4 else (3 if c <= 12 else 8)
    njp = 1 if nj == 1 else (nj + 3) // 4 * 4
    zr = 4 * njp
    nv = (nj + 3) // 4
    for sidx in range(S):
        xs = sidx * dp * c
        for J in (0, nt - 1):
            for tid in range(256):
                for u in range(nv):
                    grp = tid + 256 * u
                    if grp >= 16 * c:
                        continue
                    for i in range(4):
                        e = 4 * grp + i
                        assert 0 <= xs + J * TB * c + e < nvals
                        kk, o = divmod(e, c)
                        assert kk < TB and 0 <= kk * zr + (o & 3) * njp + (o >> 2) < TB * zr
        for I in (0, nt - 1):
            for tid in range(256):
                r, g = tid >> 2, tid & 3
                for j in range(nj):
                    o = g + 4 * j
                    if o < c:
                        assert 0 <= xs + (I * TB + r) * c + o < nvals
    # every value of a block has exactly one publishing thread
    owners = {}
    for tid in range(256):
        r, g = tid >> 2, tid & 3
        for j in range(nj):
            if g + 4 * j < c:
                key = (r, g + 4 * j)
                assert key not in owners
                owners[key] = tid
    assert len(owners) == TB * c
    # and exactly one polling thread
    polled = [4 * (tid + 256 * u) + i for tid in range(256) for u in range(nv) if tid + 256 * u < 16 * c
              for i in range(4)]
    assert sorted(polled) == list(range(TB * c))


def test_wait_check_leaves_every_cta_waiting_on_block_zero():
    """The check's launch: k (nt - 1) CTAs with tickets S .. S nt - 1 (S = k), so
    row 0 never runs; each CTA's first wait is on block 0 of its system."""
    for k, nt in [(5, 4), (5, 32), (1, 2)]:
        S = k
        rows = [ticket_to_row(tk, S, nt, 0) for tk in range(S, S * nt)]
        assert sorted(rows) == sorted((s, i) for s in range(S) for i in range(1, nt))
        assert all(waits_of(i, nt, 0)[0] == 0 for _, i in rows)
        finished, published, stuck = run_schedule(S, nt, S * nt, 0, seed=0, tk0=S, ncta=S * (nt - 1))
        assert finished == 0 and not published and len(stuck) == S * (nt - 1)
