"""Pins of the loop-closure reference on hand-worked maps (CPU only)."""
import numpy as np

from oracle import loopclosure as lc
from paper_2511_23030_b300 import synth

import oracle

S = 10.0  # chunk size


def _cam():
    return synth.Camera(100.0, 100.0, 100.0, 100.0, 200, 200, np.eye(4, dtype=np.float32))


def _rows(pts):
    r = np.zeros((len(pts), 11), np.float32)  # degree 0: 11 components
    r[:, :3] = pts
    r[:, 6] = 1.0  # identity quaternion
    r[:, 10] = np.arange(len(pts))  # tag each Gaussian through its opacity logit
    return r


def _key(p):
    return int(oracle.chunk_keys(np.asarray([p], np.float32), S)[1][0])


def _shift(dx):
    C = np.eye(4, dtype=np.float32)
    C[0, 3] = dx
    return C


def test_hand_worked_redistribution():
    # chunk x in [-5, 5): g1 (x=1), g2 (x=4), g3 (x=-3); chunk x in [5, 15): h1 (x=6), h2 (x=14); all at z = 20
    A = _rows([(1, 0, 20), (4, 0, 20), (-3, 0, 20)])
    B = _rows([(6, 0, 20), (14, 0, 20)])
    B[:, 10] += 10
    kA, kB = _key((0, 0, 20)), _key((6, 0, 20))
    new, nt, nm = lc.loop_closure({kA: A, kB: B}, S, 100.0, [_cam()], [_shift(3.0)])
    assert (nt, nm) == (5, 2)
    kC = _key((17, 0, 20))
    assert sorted(new) == sorted([kA, kB, kC])
    # A keeps g1, g3 in stored order; B keeps h1 and receives g2 after it; h2 founds a new chunk
    assert list(new[kA][:, 10]) == [0, 2] and list(new[kA][:, 0]) == [4, 0]
    assert list(new[kB][:, 10]) == [10, 1] and list(new[kB][:, 0]) == [9, 7]
    assert list(new[kC][:, 10]) == [11] and new[kC][0, 0] == 17
    assert np.array_equal(new[kA][:, 6:10], np.tile([1, 0, 0, 0], (2, 1)))


def test_global_mask_first_keyframe_wins_and_hidden_gaussians_stay():
    A = _rows([(1, 0, 20), (1, 0, -20)])  # the second is behind the camera
    kA = _key((1, 0, 20))
    kB = _key((1, 0, -20))
    maps = {kA: A[:1], kB: A[1:]}
    for order, want in (([3.0, -2.0], 4.0), ([-2.0, 3.0], -1.0)):
        new, nt, nm = lc.loop_closure(maps, S, 100.0, [_cam(), _cam()], [_shift(order[0]), _shift(order[1])])
        assert nt == 1 and nm == 0
        assert new[kA][0, 0] == want
        assert np.array_equal(new[kB], A[1:])  # not visible: untouched


def test_rotation_moves_the_rotation_and_conserves_gaussians():
    rng = np.random.default_rng(0)
    pts = np.column_stack([rng.uniform(-30, 30, 400), rng.uniform(-30, 30, 400), rng.uniform(2, 60, 400)])
    rows = _rows(pts)
    q = rng.normal(size=(400, 4)).astype(np.float32)
    rows[:, 6:10] = q
    maps = {}
    for r in rows:
        maps.setdefault(_key(r[:3]), []).append(r)
    maps = {k: np.array(v) for k, v in maps.items()}
    ang = np.deg2rad(5.0)
    C = np.eye(4, dtype=np.float32)
    C[:3, :3] = [[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]]
    C[:3, 3] = (0.5, -1.0, 0.25)
    new, nt, nm = lc.loop_closure(maps, S, 100.0, [_cam()], [C])
    allrows = np.concatenate(list(new.values()))
    assert allrows.shape[0] == 400 and nt > 50 and nm > 0
    tags = np.sort(allrows[:, 10])
    assert np.array_equal(tags, np.arange(400))
    moved = allrows[np.abs(allrows[:, 6:10] - q[allrows[:, 10].astype(int)]).max(1) > 0]
    for r in moved[:20]:
        q0 = q[int(r[10])].astype(np.float64)
        R0 = synth_rot(q0)
        R1 = synth_rot(r[6:10].astype(np.float64))
        assert np.allclose(R1, C[:3, :3] @ R0, atol=1e-6)
        p0 = pts[int(r[10])]
        assert np.allclose(r[:3], C[:3, :3] @ p0 + C[:3, 3], atol=1e-4)
    for k, rows_k in new.items():  # every Gaussian sits in the chunk of its (corrected) centre
        if rows_k.shape[0]:
            assert np.all(oracle.chunk_keys(rows_k[:, :3], S)[1] == k)


def synth_rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
