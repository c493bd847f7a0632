"""Timing invariants of the single-pass smoother's shared-memory pipeline
(`fused_smooth` in csrc/msrcg_solve.cu), checked on the CPU.

The kernel streams the rows of T_x, T_y, rp (and z and r when post-smoothing)
of one column strip into shared-memory rings with cp.async, one commit group
(two rows) per pipeline step, and before each step's barrier waits for all
but the newest W groups.  Stage q (the q-th red/black half-sweep) updates rows
2s - 3q and 2s - 3q + 1 at step s: at column i the row 2s - 3q + (i & 1), the
cell of the colour that half-sweep q updates there.  Pre-smoothing forms
t = rp - A z on rows 2s - 3S and 2s - 3S + 1; post-smoothing writes rows
2s - 3S + 1 and 2s - 3S + 2 back and adds r . z over the last stage's two rows.
This model replays the schedule's copies, ring writes and ring reads with the
kernel's constants (read from the source) for both column parities and checks
that

  1. every read finds the row it needs in its ring slot;
  2. a row copied from global memory has been waited for by the step that
     reads it;
  3. no copy lands in a slot whose row is still read: a copy issued at the
     top of step s may land while slower threads still compute step s - 1.

It also flags a wait one group shorter (post-smoothing's stage 0 reads the z
row above its pair, loaded from global memory), rings shallower than each
mode needs, and a prefetch distance under which post-smoothing would never
load the r rows of its first steps.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_math_9809043_gb300", "csrc", "msrcg_solve.cu")


def kernel_constants():
    src = open(SRC).read()
    ahead = int(re.search(r"constexpr int kFuseAhead = (\d+);", src).group(1))
    wait = re.search(r'cp\.async\.wait_group %0;\\n" ::"n"\(([^)]*)\)', src).group(1)
    depth = re.search(r"int fuse_depth\(int S\) \{ return ([^;]+); \}", src).group(1)
    rdepth = re.search(r"int fuse_rdepth\(\) \{ return ([^;]+); \}", src).group(1)
    env = {"kFuseAhead": ahead}
    return (ahead, eval(wait, env), lambda S: eval(depth, dict(env, S=S)), eval(rdepth, env))


def replay(m, ny, pre, ahead, wait, depth, rdepth):
    """Violations of the three invariants for one strip of `ny` rows."""
    S = 2 * m + 1
    D, DR = depth(S), rdepth
    lag = 3 * S if pre else 3 * S - 1
    s_end = (ny - 1 + lag) // 2
    bad = []
    # ring -> slot -> (row, group of its copy or None when computed in place);
    # the z slot of row -1 (below the strip) holds zeros until a row lands
    rings = {"cell": {}, "face": {}, "z": {D - 1: (-1, None)}, "r": {}}
    issues = {}

    def issue(step, ring, slot, row, group):
        issues.setdefault(step, []).append((ring, slot, row, group))

    # the preload issues groups 0 .. ahead-1 (and face row 0) before step 0;
    # step s issues group s + ahead
    issue(-1, "face", 0, 0, 0)
    g = 0
    while 2 * g <= ny:
        step = g - ahead if g >= ahead else -1
        for j in (2 * g, 2 * g + 1):
            if j < ny:
                issue(step, "cell", j % D, j, g)
                issue(step, "face", (j + 1) % D, j + 1, g)
                if not pre:
                    issue(step, "z", j % D, j, g)
            elif j == ny and not pre:
                issue(step, "z", j % D, j, g)  # the zero ghost row above the strip's end
        g += 1
    if not pre:
        for s in range(s_end + 1):
            for r in (0, 1):
                jr = 2 * (s + ahead) - 3 * (S - 1) + r
                if 0 <= jr < ny:
                    issue(s, "r", jr % DR, jr, s + ahead)

    def land(step):
        for ring, slot, row, group in issues.get(step, []):
            rings[ring][slot] = (row, group)

    def read(s, ring, row, need_copy):
        n = D if ring != "r" else DR
        slot = row % n if row >= 0 else D - 1
        have = rings[ring].get(slot)
        if have is None or have[0] != row:
            bad.append(("wrong row", s, ring, row, have))
        elif need_copy and have[1] is not None and have[1] > s + ahead - wait:
            bad.append(("copy not waited for", s, ring, row, have[1]))

    land(-1)
    land(0)
    for s in range(s_end + 1):
        land(s + 1)  # fast threads issue step s + 1's copies while others still compute step s
        if pre and 2 * s in (ny - 1, ny):
            rings["z"][ny % D] = (ny, None)  # the zero ghost row, written before the stages read it
        writes = []
        for q in range(S):
            for ib in (0, 1):  # column parity
                j = 2 * s - 3 * q + ib
                if not (0 <= j < ny):
                    continue
                read(s, "cell", j, True)
                read(s, "face", j, True)
                read(s, "face", j + 1, True)
                if not (pre and q == 0):
                    for jj in (j - 1, j, j + 1):
                        read(s, "z", jj, True)
                if not pre and q == S - 1:
                    read(s, "r", j, True)
                if pre and q == 0:
                    writes.append(j)  # stage 0 from zero claims rows 2s, 2s + 1 (both colours)
                    if 2 * s + 1 - ib < ny:
                        writes.append(2 * s + 1 - ib)
        for r in (0, 1):
            j = 2 * s - lag + r
            if 0 <= j < ny:
                if pre:  # t = rp - A z on a finished row
                    read(s, "cell", j, True)
                    read(s, "face", j, True)
                    read(s, "face", j + 1, True)
                    for jj in (j - 1, j, j + 1):
                        read(s, "z", jj, True)
                else:
                    read(s, "z", j, True)
        if not pre:  # r . z of the last stage's other-colour cells
            for r in (0, 1):
                jd = 2 * s - 3 * (S - 1) + r
                if 0 <= jd < ny:
                    read(s, "r", jd, True)
                    read(s, "z", jd, True)
        for j in writes:
            rings["z"][j % D] = (j, None)
    return bad


CONST = kernel_constants()


@pytest.mark.parametrize("pre", [True, False], ids=["pre", "post"])
@pytest.mark.parametrize("m", [1, 2, 3, 4])
@pytest.mark.parametrize("ny", [1, 2, 3, 4, 7, 40, 97, 98])
def test_pipeline_invariants_hold(m, ny, pre):
    assert replay(m, ny, pre, *CONST) == []


def test_depths_are_even():
    # a row pair never straddles the ring's end (pair offsets step by two rows)
    ahead, wait, depth, rdepth = CONST
    assert all(depth(2 * m + 1) % 2 == 0 for m in (1, 2, 3, 4)) and rdepth % 2 == 0


def test_model_flags_the_short_wait():
    ahead, wait, depth, rdepth = CONST
    assert wait == ahead - 1
    bad = replay(4, 40, False, ahead, ahead, depth, rdepth)
    assert bad and all(b[0] == "copy not waited for" and b[2] == "z" for b in bad)
    assert replay(4, 40, True, ahead, ahead, depth, rdepth) == []


def test_prefetch_distance_guard():
    ahead, wait, depth, rdepth = CONST
    # one step further ahead, m = 1's post-smoothing would miss its first r rows
    bad = replay(1, 40, False, ahead + 1, ahead, depth, rdepth + 2)
    assert bad and all(b[0] == "wrong row" and b[2] == "r" for b in bad)
    src = open(SRC).read()
    guard = re.search(r"bool fuse_on\(const msrcg_hier\* h\) \{ return ([^;]+); \}", src).group(1)
    assert "6 * h->o.m > 2 * kFuseAhead - 1" in guard
    assert all(6 * m > 2 * ahead - 1 for m in (1, 2, 3, 4))
    assert not 6 * 1 > 2 * (ahead + 1) - 1
    assert src.count("fuse_on(h)") == 2  # shared-memory sizing and the problem descriptor


def test_model_flags_a_shallower_ring():
    ahead, wait, depth, rdepth = CONST
    # pre-smoothing reads each row until its residual step, longer than
    # post-smoothing: one row less breaks pre, three rows less break post
    assert any(b[0] == "wrong row" for b in replay(4, 97, True, ahead, wait, lambda S: depth(S) - 1, rdepth))
    assert replay(4, 97, False, ahead, wait, lambda S: depth(S) - 2, rdepth) == []
    assert any(b[0] == "wrong row" for b in replay(4, 97, False, ahead, wait, lambda S: depth(S) - 3, rdepth))
    bad = replay(4, 97, False, ahead, wait, depth, rdepth - 1)
    assert any(b[0] == "wrong row" and b[2] == "r" for b in bad)
