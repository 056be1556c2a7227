"""Host logic of the persistent batched schedule: the plan of teams and the work queue.

The plan is computed on the host from the sizes alone (gf2_batch_plan exports it, no device
call), so its invariants are checked here on a CPU: teams are disjoint contiguous CTA ranges of
power-of-two size, every matrix is either in exactly one team or in the queue, and the sizes of
the workloads decide the automatic schedule as documented (the 2048-matrix batch has no team
above 16 CTAs and runs persistently; a 65536 x 65536 member gets a larger team and sends the
call to the per-step schedule).
"""
from __future__ import annotations

import pytest

from paper_1006_1744_gb300 import synth as S

SM = 152


@pytest.fixture(scope="module")
def gf2():
    from paper_1006_1744_gb300 import build, gf2
    build.build()
    return gf2


def check_plan(shapes, ctas, plan):
    team_of, sizes, member = plan
    nt = len(sizes)
    assert len(team_of) == ctas and len(member) == len(shapes)
    for t, g in enumerate(sizes):
        assert g >= 2 and g & (g - 1) == 0, (t, g)
        ctas_t = [c for c in range(ctas) if team_of[c] == t]
        assert len(ctas_t) == g
        assert ctas_t == list(range(ctas_t[0], ctas_t[0] + g)), "team CTAs must be contiguous"
    assert all(-1 <= x < nt for x in team_of)
    assert sum(sizes) == sum(1 for x in team_of if x >= 0) <= ctas
    assert all(-1 <= x < nt for x in member)
    for t in range(nt):
        assert any(x == t for x in member), f"team {t} has no matrix"


def test_config4_batch_plan(gf2):
    """The 2048-matrix batch: no member is worth a team larger than 16 CTAs (the automatic
    choice is the persistent launch); in fact the largest member's one-CTA cost stays under the
    average load per CTA, so every matrix comes from the work queue."""
    shapes = [(m, n) for (m, n, p, sd) in S.batch_recipe(2048, 0x10061744)]
    plan = gf2.batch_plan(shapes, SM)
    check_plan(shapes, SM, plan)
    team_of, sizes, member = plan
    assert max(sizes, default=1) <= 16
    assert gf2.batch_plan(shapes, SM) == plan  # deterministic


def test_mixed_batch_teams_take_the_large_members(gf2):
    shapes = [(1024, 1024)] * 400 + [(16384, 16384)] * 4 + [(2048, 4096)] * 50
    plan = gf2.batch_plan(shapes, SM)
    check_plan(shapes, SM, plan)
    team_of, sizes, member = plan
    assert sizes, "the 16384^2 members must get teams"
    assert all(member[i] >= 0 for i in range(400, 404))
    assert all(member[i] == -1 for i in range(400))
    assert any(x == -1 for x in team_of)       # queue workers remain for the small ones


def test_one_huge_member_gets_a_large_team(gf2):
    shapes = [(65536, 65536)] + [(512, 512)] * 64
    plan = gf2.batch_plan(shapes, SM)
    check_plan(shapes, SM, plan)
    team_of, sizes, member = plan
    assert member[0] >= 0 and sizes[member[0]] > 16   # automatic choice: per-step schedule
    assert all(x == -1 for x in member[1:])


def test_small_matrices_all_queued(gf2):
    shapes = [(256, 256)] * 500 + [(64, 64)] * 10
    team_of, sizes, member = gf2.batch_plan(shapes, SM)
    assert sizes == [] and all(x == -1 for x in team_of) and all(x == -1 for x in member)


@pytest.mark.parametrize("ctas", [1, 2, 7, 64, 152, 1024])
def test_plan_any_grid(gf2, ctas):
    shapes = [(m, n) for (m, n, p, sd) in S.batch_recipe(300, 7)] + [(16384, 16384)]
    check_plan(shapes, ctas, gf2.batch_plan(shapes, ctas))


def test_plan_rejects_bad_arguments(gf2):
    with pytest.raises(gf2.Gf2Error):
        gf2.batch_plan([(64, 64)], 0)
    with pytest.raises(gf2.Gf2Error):
        gf2.batch_plan([(64, 64)], 1025)
    with pytest.raises(gf2.Gf2Error):
        gf2.batch_plan([(-1, 64)], 8)
