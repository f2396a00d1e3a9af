"""Host arithmetic of the batched sliding join, without a GPU: the groups
of windows cover every window once and in order, each group's panes are its
windows' panes (window w: panes w .. w + per - 1), and the host copies tile
the rows in order, every row of a group's panes copied by the group's turn."""
import pytest

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("nwin,per,groups", [(509, 4, 8), (9, 4, 4), (1, 4, 8), (3, 2, 8), (100, 1, 7), (64, 8, 16),
                                             (10, 4, 1)])
def test_window_groups_cover_windows_and_rows(nwin, per, groups):
    from paper_1901_01328_b300.pipeline import window_groups
    stride = 250
    grp = window_groups(nwin, per, stride, groups)
    assert 1 <= len(grp) <= min(groups, nwin)
    assert grp[0][0] == 0 and grp[-1][1] == nwin
    for a, b in zip(grp, grp[1:]):
        assert a[1] == b[0]
    done = 0
    for w0, w1, p0, p1, c0, c1 in grp:
        assert w0 < w1
        assert (p0, p1) == (w0, w1 + per - 1)
        assert c0 == done and c1 == p1 * stride and p0 * stride <= c1
        done = c1
    assert done == (nwin + per - 1) * stride
