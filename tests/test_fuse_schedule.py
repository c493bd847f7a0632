"""Timing invariants of the single-pass smoother's shared-memory pipeline
(`fused_smooth` in csrc/msrcg_solve.cu), checked on the CPU.

The kernel streams the rows of T_x, T_y, rp (and z and r when post-smoothing)
of one column strip into shared-memory rings with cp.async, one commit group
per pipeline step, and before each step's barrier waits for all but the
newest W groups.  Stage q (the q-th red/black half-sweep) updates row s - 2q
at step s.  This model replays the schedule's copies, ring writes and ring
reads with the kernel's constants (read from the source) and checks that

  1. every read finds the row it needs in its ring slot;
  2. a row copied from global memory has been waited for by the step that
     reads it;
  3. no copy lands in a slot whose row is still read: a copy issued at the
     top of step s may land while slower threads still compute step s - 1.

The library runs the pipeline for smoothing degrees m = 2..4 (the paper's
m = 4 by default); for m = 1 post-smoothing would never load the first r
rows, which the model flags and the host keeps off the single pass.  The
model also flags a wait one group shorter, the defect the GPU determinism
test once found (post-smoothing's stage 0 read the z row above its own
before that row's copy had been waited for), and rings shallower than each
mode needs.
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
    lag = 2 * S if pre else 2 * S - 1
    s_end = ny - 1 + lag
    bad = []
    # ring -> slot -> (row, group of its copy or None when computed in place)
    rings = {"cell": {}, "face": {}, "z": {D - 1: (-1, None)}, "r": {}}
    # copies per issuing step: (ring, slot, row, group); the preload issues
    # groups 0 .. ahead-1 before step 0
    issues = {}

    def issue(step, ring, slot, row, group):
        issues.setdefault(step, []).append((ring, slot, row, group))

    issue(-1, "face", 0, 0, 0)
    for jl in range(ny + 1):
        step = jl - ahead if jl >= ahead else -1
        if jl < ny:
            issue(step, "cell", jl % D, jl, jl)
            issue(step, "face", (jl + 1) % D, jl + 1, jl)
            if not pre:
                issue(step, "z", jl % D, jl, jl)
        elif not pre:
            issue(step, "z", jl % D, jl, jl)  # the zero ghost row below the strip's end
    if not pre:
        for s in range(s_end + 1):
            jr = s + ahead - 2 * (S - 1)
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
        if pre and s == ny:
            rings["z"][ny % D] = (ny, None)  # the zero ghost row, written before the stages read it
        writes = []
        for q in range(S):
            j = s - 2 * q
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
                writes.append(j)  # stage 0 from zero claims row j's z slot
        j = s - lag
        if 0 <= j < ny:
            if pre:  # t = rp - A z on the finished row
                read(s, "cell", j, True)
                read(s, "face", j, True)
                read(s, "face", j + 1, True)
                for jj in (j - 1, j, j + 1):
                    read(s, "z", jj, True)
            else:
                read(s, "z", j, True)
        jd = s - 2 * (S - 1)
        if not pre and 0 <= jd < ny:
            read(s, "r", jd, True)
        for j in writes:
            rings["z"][j % D] = (j, None)
    return bad


CONST = kernel_constants()


@pytest.mark.parametrize("pre", [True, False], ids=["pre", "post"])
@pytest.mark.parametrize("m", [2, 3, 4])
@pytest.mark.parametrize("ny", [1, 2, 3, 7, 40, 97])
def test_pipeline_invariants_hold(m, ny, pre):
    assert replay(m, ny, pre, *CONST) == []


def test_model_flags_the_short_wait():
    ahead, wait, depth, rdepth = CONST
    assert wait == ahead - 1
    bad = replay(4, 40, False, ahead, ahead, depth, rdepth)
    assert bad and all(b[0] == "copy not waited for" and b[2] == "z" for b in bad)
    assert replay(4, 40, True, ahead, ahead, depth, rdepth) == []


def test_m1_stays_off_the_single_pass():
    ahead, wait, depth, rdepth = CONST
    bad = replay(1, 40, False, ahead, wait, depth, rdepth)
    assert bad and all(b[0] == "wrong row" and b[2] == "r" for b in bad)
    src = open(SRC).read()
    guard = re.search(r"bool fuse_on\(const msrcg_hier\* h\) \{ return ([^;]+); \}", src).group(1)
    assert "4 * h->o.m >= kFuseAhead" in guard
    assert src.count("fuse_on(h)") == 2  # shared-memory sizing and the problem descriptor


def test_model_flags_a_shallower_ring():
    ahead, wait, depth, rdepth = CONST
    # pre-smoothing reads each row until its residual step, two steps longer
    # than post-smoothing: one row less breaks pre, three rows less break post
    assert any(b[0] == "wrong row" for b in replay(4, 97, True, ahead, wait, lambda S: depth(S) - 1, rdepth))
    assert replay(4, 97, False, ahead, wait, lambda S: depth(S) - 2, rdepth) == []
    assert any(b[0] == "wrong row" for b in replay(4, 97, False, ahead, wait, lambda S: depth(S) - 3, rdepth))
    bad = replay(4, 97, False, ahead, wait, depth, rdepth - 1)
    assert any(b[0] == "wrong row" and b[2] == "r" for b in bad)
