"""Checks of a level tree (Fig. 2 of the paper): the entries (level, call,
iterations, pass) of every PCG call of every level, in the order the calls
returned.  Shared by the oracle pins and the GPU tests."""


def check_tree(entries, iters, calls, nlev, coarsest_exact=True):
    """The structure the recursion of eq. 2.10 fixes: every CG iteration of
    level k applies the preconditioner once, which calls level k+1's PCG
    once, and a call returns after the calls it made.  So the level-(k+1)
    entries returned since the previous level-k entry are as many as that
    level-k call's iterations; per level the entries number the calls
    0, 1, ... and add up to the level's iteration counter; the coarsest
    level's exact inverse ends each of its calls after one iteration."""
    pending = [0] * (nlev + 1)  # level-(k+1) entries since the last level-k entry
    seen = [0] * nlev
    total = [0] * nlev
    for lev, call, it, _pass in entries:
        assert 0 <= lev < nlev, (lev, nlev)
        assert call == seen[lev], (lev, call, seen[lev])  # calls in order
        seen[lev] += 1
        total[lev] += it
        if lev < nlev - 1:
            assert pending[lev] == it, ("children of a call", lev, call, pending[lev], it)
        elif coarsest_exact:
            assert it in (0, 1), ("coarsest call", call, it)
        pending[lev] = 0
        if lev > 0:
            pending[lev - 1] += 1
    assert seen == list(calls[:nlev]), (seen, calls)
    assert total == list(iters[:nlev]), (total, iters)
    assert all(v == 0 for v in pending[:nlev])
    # the outermost level's calls are the passes of the solve
    assert [e[3] for e in entries if e[0] == 0] == list(range(seen[0]))
