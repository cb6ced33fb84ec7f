"""The backprojection's grouping of slices one or more pitches apart (host logic, no GPU).

By the periodicity of Sec. II a slice m pitches up sees view k + m views_per_turn exactly as the
slice m pitches down sees view k, so the multi-pitch kernel reconstructs groups of slices one pitch
apart together.  The grouping must put every slice of a launch in exactly one place (an item group
or a one-group range), within the forms the library instantiates."""
import pytest

from paper_2201_02309_b300 import build, native

FORMS = {4: {8, 6}, 3: {10, 8}, 2: {14, 12}}


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()


def covered(items, rest, N):
    out = []
    for G, T, s0, cnt in items:
        for m in range(G):
            out += range(s0 + m * N, s0 + m * N + cnt)
    for s, e in rest:
        out += range(s, e)
    return out


@pytest.mark.parametrize("S0,S1,N,gmax", [(0, 256, 70, 4), (0, 256, 70, 3), (0, 256, 70, 2), (48, 194, 58, 4),
                                          (0, 194, 58, 4), (0, 150, 58, 4), (16, 32, 58, 4), (0, 1000, 70, 4),
                                          (0, 69, 70, 4), (0, 70, 70, 4), (0, 71, 70, 4), (64, 256, 70, 4),
                                          (0, 23, 5, 4), (0, 300, 7, 3), (32, 33, 1, 2)])
def test_every_slice_once(S0, S1, N, gmax):
    items, rest = native.katsevich_slice_groups(S0, S1, N, gmax)
    got = covered(items, rest, N)
    assert sorted(got) == list(range(S0, S1)), "a slice missing or taken twice"
    for G, T, s0, cnt in items:
        assert 2 <= G <= gmax and T in FORMS[G] and 1 <= cnt <= T
        assert S0 <= s0 and s0 + (G - 1) * N + cnt <= S1
    for s, e in rest:
        assert S0 <= s < e <= S1


def test_clinical_volume_grouping():
    """512 x 512 x 256 at 70 slices per pitch: slices 0-45 lead four groups (five items of 8 and
    one of 6), 46-69 three (three items of 8); nothing is left to the one-group kernel."""
    items, rest = native.katsevich_slice_groups(0, 256, 70, 4)
    assert rest == []
    assert items == [(4, 8, s, 8) for s in range(0, 40, 8)] + [(4, 6, 40, 6)] + [(3, 8, s, 8) for s in (46, 54, 62)]


def test_two_group_limit_splits_four_pitches():
    """With at most two groups per item, four pitches split into two pairs per leading slice, and
    of three pitches the third goes to the one-group kernel."""
    items, rest = native.katsevich_slice_groups(0, 256, 70, 2)
    assert rest == [(186, 210)]
    assert all(G == 2 for G, _, _, _ in items)
    leads = sorted({s0 for _, _, s0, _ in items})
    assert 0 in leads and 140 in leads and 70 not in leads


def test_one_pitch_or_less_is_one_group():
    items, rest = native.katsevich_slice_groups(16, 80, 70, 4)
    assert items == [] and rest == [(16, 80)]


def test_bad_arguments():
    for args in [(10, 5, 70, 4), (0, 10, 0, 4), (0, 10, 70, 5), (0, 10, 70, 1), (-1, 10, 70, 4)]:
        with pytest.raises(native.KatsevichError) as e:
            native.katsevich_slice_groups(*args)
        assert e.value.status == native.KATS_EINVAL


@pytest.mark.parametrize("S0,S1,N", [(80, 256, 70), (64, 256, 70), (0, 256, 70), (48, 194, 58), (16, 300, 7),
                                     (0, 141, 70)])
def test_groups_of_leads_partition_the_slab(S0, S1, N):
    """The host pipeline's last slab in groups of leading slices [la, lb): each launch over [la, S1)
    restricted to leads below lb.  Over any partition of the leads into such groups, every slice of
    the slab is reconstructed exactly once."""
    le = min(S0 + N, S1)
    for cuts in ([S0, le], [S0, (S0 + le) // 2, le], list(range(S0, le, 5)) + [le]):
        got = []
        for la, lb in zip(cuts[:-1], cuts[1:]):
            items, rest = native.katsevich_slice_groups(la, S1, N, 4, lb)
            got += covered(items, rest, N)
        assert sorted(got) == list(range(S0, S1)), cuts
