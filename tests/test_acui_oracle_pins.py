"""Pins of the FP64 ACUI oracle (Eq. 13) against facts outside it, and the host-side point
count of the C ABI against it (no device calls)."""
import itertools

import numpy as np
import pytest

from oracle import acui64 as A


def test_paper_setting_count_by_hand():
    # d = 8 on a 256-voxel axis: floor(256 / 16) + 1 = 17, so n runs over -17..17: 35 points
    assert A.half_count(256, 8) == 17
    assert A.acui_count((200.0, 200.0, 200.0), (256, 256, 256), 8) == 35 ** 3
    # a non-integer interval: 100 / 7 = 14.28..., floor 14, plus one; 10 / 7 -> 1 + 1;
    # 1 / 7 -> 0 + 1: a one-voxel axis still gets -1, 0, 1
    assert A.half_count(100, 3.5) == 15
    assert A.acui_count((1.0, 2.0, 3.0), (100, 10, 1), 3.5) == 31 * 5 * 3


def test_points_equal_a_brute_force_enumeration():
    S, M, d = (30.0, 50.0, 70.0), (12, 9, 5), 2
    want = set()
    for n in itertools.product(range(-20, 21), repeat=3):
        # the inequality of Eq. 13 with the integer floor of M / (2 d) for integer d
        if all(-(m // (2 * d)) - 1 <= k <= m // (2 * d) + 1 for k, m in zip(n, M)):
            want.add(tuple(round(k * s * d / m, 9) for k, s, m in zip(n, S, M)))
    got = A.acui_points64(S, M, d)
    assert got.shape[1] == len(want)
    assert {tuple(round(x, 9) for x in p) for p in got.T} == want


def test_grid_is_centred_uniform_and_overhangs_the_cuboid():
    S, M, d = (120.0, 80.0, 200.0), (64, 100, 37), 8
    P = A.acui_points64(S, M, d)
    np.testing.assert_allclose(P.mean(axis=1), 0.0, atol=1e-9)
    for a in range(3):
        vals = np.unique(P[a])
        h = S[a] * d / M[a]
        np.testing.assert_allclose(np.diff(vals), h, rtol=1e-12)
        assert 0.0 in vals
        # the outermost points reach at least half the cuboid side, and at most one spacing beyond
        assert S[a] / 2 - 1e-9 <= vals.max() <= S[a] / 2 + 2 * h
        assert vals.min() == -vals.max()


def test_ordering_n1_slowest():
    P = A.acui_points64((10.0, 10.0, 10.0), (8, 8, 8), 2)  # 8 / 4 = 2: n in -3..3, 7 per axis
    assert P.shape == (3, 343)
    assert (np.diff(P[2][:7]) > 0).all() and (P[0][:49] == P[0][0]).all()
    assert P[0][0] < P[0][49] and P[1][0] < P[1][7]
    np.testing.assert_allclose(P[:, 0], [-7.5, -7.5, -7.5])  # -3 * 10 * 2 / 8


def test_host_count_of_the_library_matches_the_oracle():
    from paper_2403_04116_gb300 import binding as B
    B.lib(build_if_missing=True)
    for S, M, d in [((200.0,) * 3, (256,) * 3, 8), ((1.0, 2.0, 3.0), (100, 10, 1), 3.5), ((5.0,) * 3, (1, 1, 1), 0.25),
                    ((7.0, 9.0, 11.0), (13, 17, 19), 1.0)]:
        assert B.xg_acui_count(S, M, d) == A.acui_count(S, M, d)
    for bad in [((0.0, 1.0, 1.0), (8, 8, 8), 2), ((1.0,) * 3, (0, 8, 8), 2), ((1.0,) * 3, (8, 8, 8), 0.0),
                ((1.0,) * 3, (8, 8, 8), float("nan")), ((1.0,) * 3, (1 << 30,) * 3, 1.0)]:
        assert B.xg_acui_count(*bad) == 0


def test_projection_noise_level():
    from paper_2403_04116_gb300 import synth
    gen = np.random.default_rng(0)
    img = np.stack([np.linspace(0.0, 2.0, 40000).reshape(200, 200), np.full((200, 200), 0.5)])
    img[1, 0, 0] = 1.5  # value range 1
    noisy = synth.projection_noise(img, 0.03, gen)
    assert np.std(noisy[0] - img[0]) == pytest.approx(0.06, rel=0.03)
    assert np.std(noisy[1] - img[1]) == pytest.approx(0.03, rel=0.03)
    assert abs(np.mean(noisy - img)) < 1e-3
