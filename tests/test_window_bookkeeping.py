"""Host-side index simulation of the solver's basis bookkeeping (no GPU).

The iteration of `Engine::run` (paper_2111_06552_gb300/csrc/solver.cu) writes the next
basis [X_a | P | W] into a row-major buffer of width dmax = sizeX + 2 bs, starting
at column xoff.  With the moving mechanism (Section 3.3) and, in the FP64 phase of
the mixed path, a reservoir of phase-1 vectors that refills the window beside W,
the column counts vary from iteration to iteration.  This test replays the
bookkeeping with random outcomes of every data-dependent step (converged prefix,
columns kept by STEP 2 and STEP 5, move decisions) and checks that every block the
iteration writes stays inside the buffer.  Its formulas restate the ones in
`Engine::run`; a change there must be mirrored here.
"""
import random


def _simulate(rng, size_x, bs, nev, moving, nres, iters=400):
    dmax = size_x + 2 * bs
    ldW = -(-max(size_x, 2 * bs) // 4) * 4
    kx, npn_prev, nw = size_x, 0, 0
    nlock, lw, res_next, kgrow = 0, 0, size_x if nres else 0, 0
    first = True
    for _ in range(iters):
        d = kx + npn_prev + nw
        assert 0 < d <= dmax
        if kgrow > 0:
            kx = min(kx + kgrow, d)
            kgrow = 0
        # X_new = V_a x^ writes kx columns at offset 0 of the other buffer
        assert kx <= dmax
        c = rng.randint(0, kx)                      # converged prefix (STEP 4)
        reservoir_left = nres and res_next < nres
        move = (not reservoir_left) and moving and nlock + c < nev and (lw + c >= 2 * bs or c == kx)
        nlock += c
        if nlock >= nev:
            return
        xoff, kxn, npn = c, kx - c, 0
        if move:
            kxn = min(size_x, d - c)
            xoff, lw = 0, 0
        else:
            lw += c
        bsn = min(bs, nev - nlock, kxn)
        if not move and not first and bsn > 0:
            npn = rng.randint(0, bsn)               # P columns kept (STEP 5)
        rres = 0
        if nres and res_next < nres and kxn < size_x:
            rres = min(nres - res_next, size_x - kxn)
            rres = min(rres, ldW - bsn)
            if xoff > 0 and xoff + kxn + npn + bsn + rres > dmax:
                # [X_a, P] move to column 0 (staged through a buffer of width ldW)
                assert kxn <= ldW and npn <= ldW
                xoff = 0
            rres = min(rres, dmax - (xoff + kxn + npn + bsn))
            rres = max(rres, 0)
            res_next += rres
        # reservoir vectors are staged beside W's bsn columns in a buffer of width ldW
        assert bsn + rres <= ldW
        nwn = rng.randint(0, bsn + rres)           # W columns kept (STEP 2)
        kgrow = rres
        assert xoff + kxn + npn + nwn <= dmax      # the next basis fits the buffer
        if kxn + npn + nwn == 0:
            return
        kx, npn_prev, nw = kxn, npn, nwn
        first = False


def test_basis_never_exceeds_buffer():
    rng = random.Random(12345)
    runs = 0
    for _ in range(3000):
        bs = rng.randint(1, 12)
        moving = rng.random() < 0.7
        nev = rng.randint(bs, 20 * bs)
        size_x = 3 * bs if moving else nev + 3 * bs
        nres = rng.choice([0, 0, rng.randint(size_x, nev + size_x)])
        _simulate(rng, size_x, bs, nev, moving, nres)
        runs += 1
    assert runs == 3000


def test_old_refill_bound_overflowed():
    """The refill bound without the basis offset (columns already used by X_a and P)
    lets W run past the buffer; the simulation must see that, else it proves nothing."""
    rng = random.Random(7)
    hit = 0
    for _ in range(2000):
        bs = rng.randint(2, 8)
        size_x, nev = 3 * bs, 12 * bs
        dmax = size_x + 2 * bs
        kxn = rng.randint(1, size_x - 1)
        xoff = rng.randint(0, size_x - kxn)
        npn = rng.randint(0, bs)
        bsn = bs
        rres_old = size_x - kxn                     # bounded by the window only
        nwn = bsn + rres_old                        # every staged column kept
        if xoff + kxn + npn + nwn > dmax:
            hit += 1
    assert hit > 0


def test_refill_keeps_the_window_full():
    """With P and W at full width, pairs that lock free window slots at the front of
    the buffer; the refill must still reach them (the window does not shrink while
    phase-1 vectors are left)."""
    bs, nev = 4, 40
    size_x = 3 * bs
    dmax, ldW = size_x + 2 * bs, size_x
    kx, c, npn, bsn = size_x, 3, bs, bs
    xoff, kxn = c, kx - c
    rres = min(100, size_x - kxn, ldW - bsn)
    if xoff > 0 and xoff + kxn + npn + bsn + rres > dmax:
        xoff = 0
    rres = min(rres, dmax - (xoff + kxn + npn + bsn))
    assert kxn + rres == size_x
