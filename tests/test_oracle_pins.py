"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a worked example, a closed form, an
invariant, or brute-force enumeration on a tiny grid (``bruteforce.py``,
which shares no code with the oracle).  The tests are chosen so that a
dropped term, a wrong sign, a wrong index or a transposed operand in the
oracle fails at least one of them (``test_planted_mistakes_fail_replan_pin``
compiles copies of the oracle with such mistakes and checks that they fail).
"""
import os
from fractions import Fraction
from math import floor

import numpy as np
import pytest

import bruteforce as BF
import oracle as O
import scenegen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_scene(rng, shape, n_boxes, side_hi, keep=()):
    nx, ny, nz = shape
    boxes = []
    while len(boxes) < n_boxes:
        s = rng.integers(1, side_hi + 1, 3)
        c = rng.integers(0, [nx, ny, nz])
        b = [int(c[0]), int(c[1]), int(c[2]), int(c[0] + s[0] - 1), int(c[1] + s[1] - 1),
             int(c[2] + s[2] - 1)]
        if any(all(b[a] <= p[a] <= b[a + 3] for a in range(3)) for p in keep):
            continue
        boxes.append(b)
    return np.asarray(boxes, np.int32).reshape(-1, 6)


# --------------------------------------------------------------------- shells

def test_shell_bounds_closed_form():
    # tol = 1/2 with integer L: (L - 1/2)^2 = L^2 - L + 1/4, (L + 1/2)^2 = L^2 + L + 1/4
    for L in range(1, 40):
        assert O.shell_bounds(L, 0.5) == (L * L - L + 1, L * L + L)


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8, 13, 20])
def test_shell_matches_mesh_and_order(L):
    lo, hi = O.shell_bounds(L)
    sh = O.shell(lo, hi)
    ref = BF.shell_offsets(lo, hi)
    assert set(map(tuple, sh.tolist())) == set(map(tuple, ref.tolist()))
    assert len(sh) == len(ref)
    key = [(int(d @ d), int(d[2]), int(d[1]), int(d[0])) for d in sh.astype(np.int64)]
    assert key == sorted(key)


def test_shell_symmetric():
    lo, hi = O.shell_bounds(7)
    s = set(map(tuple, O.shell(lo, hi).tolist()))
    assert s == {(-a, -b, -c) for a, b, c in s}
    assert s == {(b, c, a) for a, b, c in s}


# ----------------------------------------------------------------- supercover

def test_supercover_worked_examples():
    with open(os.path.join(GOLDEN, "supercover_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seg, vox = line.split("|")
            a_b = [int(v) for v in seg.split()]
            want = {tuple(int(v) for v in t.split()) for t in vox.split(";")}
            got = set(map(tuple, O.supercover(a_b[:3], a_b[3:]).tolist()))
            assert got == want, line


def test_supercover_vs_chebyshev_every_small_offset():
    for lo, hi in [(1, 12), (13, 30)]:
        for d in BF.shell_offsets(lo, hi):
            d = tuple(int(v) for v in d)
            got = set(map(tuple, O.supercover((0, 0, 0), d).tolist()))
            assert got == set(BF.supercover_from_origin(d)), d


def test_supercover_vs_chebyshev_random_segments():
    rng = np.random.default_rng(7)
    for _ in range(300):
        a = tuple(int(v) for v in rng.integers(-6, 7, 3))
        b = tuple(int(v) for v in rng.integers(-6, 7, 3))
        got = set(map(tuple, O.supercover(a, b).tolist()))
        assert got == set(BF.supercover(a, b)), (a, b)


def test_supercover_translation_and_reversal():
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = rng.integers(-20, 20, 3)
        d = rng.integers(-9, 10, 3)
        base = {tuple(v) for v in O.supercover((0, 0, 0), d).tolist()}
        moved = {tuple(v) for v in O.supercover(p, p + d).tolist()}
        assert moved == {tuple(np.asarray(v) + p) for v in base}
        back = {tuple(v) for v in O.supercover(p + d, p).tolist()}
        assert back == moved


def test_supercover_contains_endpoints_and_is_in_bbox():
    rng = np.random.default_rng(5)
    for _ in range(100):
        a = rng.integers(0, 30, 3)
        b = rng.integers(0, 30, 3)
        sc = O.supercover(a, b)
        s = set(map(tuple, sc.tolist()))
        assert tuple(a) in s and tuple(b) in s
        assert (sc >= np.minimum(a, b)).all() and (sc <= np.maximum(a, b)).all()


# ------------------------------------------------------------------ rasterize

def test_rasterize_matches_numpy_fill():
    rng = np.random.default_rng(1)
    boxes = _rand_scene(rng, (20, 17, 13), 12, 7)
    boxes[0] = [-3, -3, -3, 2, 2, 2]  # clipped at the low faces
    boxes[1] = [15, 10, 8, 40, 40, 40]  # clipped at the high faces
    occ = O.rasterize((20, 17, 13), boxes)
    assert (occ.astype(bool) == BF.occupancy((20, 17, 13), boxes)).all()


# ------------------------------------------------ sets and reach, brute force

TINY = [
    # shape, lengths, n_boxes, seed
    ((9, 8, 7), (3, 2, 2), 4, 0),
    ((8, 8, 8), (2, 3, 2), 6, 1),
    ((10, 7, 6), (3, 3), 5, 2),
    ((7, 7, 7), (2, 2, 2), 3, 3),
    ((9, 9, 5), (4, 2, 2), 5, 4),
]


@pytest.mark.parametrize("shape,lengths,n_boxes,seed", TINY)
def test_sets_and_reach_vs_enumeration(shape, lengths, n_boxes, seed):
    rng = np.random.default_rng(100 + seed)
    nx, ny, nz = shape
    root = (nx // 2, ny // 2, 0)
    boxes = _rand_scene(rng, shape, n_boxes, 3, keep=[root])
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    ch = BF.Chains(BF.occupancy(shape, boxes), bounds)
    F = O.forward(occ, lengths, root)
    # several targets, including occupied and unreachable ones
    targets = [tuple(int(v) for v in rng.integers(0, [nx, ny, nz])) for _ in range(6)]
    targets.append(root)
    poses, found, vs = O.reach_many(occ, lengths, root, targets, want_sets=True)
    for i, t in enumerate(targets):
        Fb, Vb, good = ch.joint_sets(root, [t])
        for k in range(len(lengths) + 1):
            assert BF.to_set(F[k]) == Fb[k], ("F", k)
            assert BF.to_set(vs[i, k]) == Vb[k], ("V", t, k)
        assert bool(found[i]) == bool(good), t
        if good:
            assert tuple(map(tuple, poses[i].tolist())) == ch.lexmin(good), t


CONES = [((0, 0, 1), 1, 2), ((1, 0, 0), 0, 1), ((1, 1, 1), 1, 4), ((0, -1, 2), 3, 4),
         ((-2, 1, 1), 1, 3)]


def _cone_offsets(lo2, hi2, cone):
    """The shell's offsets inside the cone (vectorised over the numpy mesh):
    positive projection on the axis and cos^2 of the angle >= num / den."""
    (ax, ay, az), num, den = cone
    D = BF.shell_offsets(lo2, hi2).astype(np.int64)
    a = np.array([ax, ay, az], np.int64)
    proj = D @ a
    keep = (proj > 0) & (den * proj * proj >= num * (D * D).sum(1) * (a @ a))
    return D[keep]


@pytest.mark.parametrize("scene", range(len(TINY)))
def test_reach_set_and_cone_vs_enumeration(scene):
    """Target clouds with an approach cone on the last segment (section "The
    gap in gMS"): found, pose (lexicographically smallest chain) and V_k for
    k < S against enumeration of every chain whose last segment lies in the
    cone; V_S = F_S & T."""
    shape, lengths, n_boxes, seed = TINY[scene]
    rng = np.random.default_rng(500 + seed)
    nx, ny, nz = shape
    root = (nx // 2, ny // 2, 0)
    boxes = _rand_scene(rng, shape, n_boxes, 3, keep=[root])
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    ch = BF.Chains(BF.occupancy(shape, boxes), bounds)
    S = len(lengths)
    for ci, cone in enumerate(CONES + [None]):
        cloud = [tuple(int(v) for v in rng.integers(0, [nx, ny, nz])) for _ in range(4)]
        T = np.zeros(occ.shape, np.uint8)
        for t in cloud:
            T[t[2], t[1], t[0]] = 1
        last = None if cone is None else _cone_offsets(*bounds[-1], cone)
        Fb, Vb, good = ch.joint_sets(root, cloud, last_offsets=last)
        flat = None if cone is None else (*cone[0], cone[1], cone[2])
        pose, found, vs = O.reach_set(occ, lengths, root, T, flat)
        assert found == bool(good), (ci, cloud)
        if good:
            assert tuple(map(tuple, pose.tolist())) == ch.lexmin(good), ci
            for j in range(1, S):
                assert (pose[j] - pose[j - 1] != 0).any()
            if last is not None:
                d = tuple(int(v) for v in pose[S] - pose[S - 1])
                assert d in set(map(tuple, last.tolist()))
        for k in range(S):
            assert BF.to_set(vs[k]) == Vb[k], (ci, k)
        assert BF.to_set(vs[S]) == Fb[S] & BF.to_set(T), ci


def test_reach_cone_exact_axis_closed_form():
    """cos^2 = 1: the last segment is exactly L along the axis, so a chain
    exists iff the arm without its last segment reaches t - L * axis and the
    segment from there to t is free; the pose then ends with that point."""
    shape, lengths = (11, 11, 11), (3, 2, 3)
    rng = np.random.default_rng(42)
    root = (5, 5, 0)
    boxes = _rand_scene(rng, shape, 5, 3, keep=[root])
    occ = O.rasterize(shape, boxes)
    S, L = len(lengths), lengths[-1]
    hits = 0
    for _ in range(30):
        t = tuple(int(v) for v in rng.integers(0, 11, 3))
        T = np.zeros(occ.shape, np.uint8)
        T[t[2], t[1], t[0]] = 1
        pose, found, _ = O.reach_set(occ, lengths, root, T, (0, 0, -1, 1, 1))
        q = (t[0], t[1], t[2] + L)  # joint S-1 straight above t
        want = False
        if q[2] < 11 and not occ[t[2], t[1], t[0]]:
            p2, f2, _ = O.reach_many(occ, lengths[:-1], root, [q])
            seg_free = all(not occ[z, t[1], t[0]] for z in range(t[2], q[2] + 1))
            want = bool(f2[0]) and seg_free
        assert found == want, t
        if found:
            hits += 1
            assert tuple(pose[S - 1]) == q and tuple(pose[S]) == t
    assert hits > 0


def test_reach_set_union_law():
    """A cloud's solution is the better of its parts: found(T1 | T2) =
    found(T1) or found(T2), and the chosen chain is the lexicographically
    smaller of the two parts' chains."""
    shape, lengths, n_boxes, seed = TINY[0]
    rng = np.random.default_rng(77)
    nx, ny, nz = shape
    root = (nx // 2, ny // 2, 0)
    boxes = _rand_scene(rng, shape, n_boxes, 3, keep=[root])
    occ = O.rasterize(shape, boxes)
    key = lambda p: tuple(int((q[2] * ny + q[1]) * nx + q[0]) for q in p[1:])
    for cone in (None, (0, 0, 1, 1, 4)):
        for _ in range(6):
            Ts = []
            for _ in range(2):
                T = np.zeros(occ.shape, np.uint8)
                for t in rng.integers(0, [nx, ny, nz], (3, 3)):
                    T[t[2], t[1], t[0]] = 1
                Ts.append(T)
            p1, f1, _ = O.reach_set(occ, lengths, root, Ts[0], cone)
            p2, f2, _ = O.reach_set(occ, lengths, root, Ts[1], cone)
            pu, fu, _ = O.reach_set(occ, lengths, root, Ts[0] | Ts[1], cone)
            assert fu == (f1 or f2)
            if fu:
                best = min([p for p, f in ((p1, f1), (p2, f2)) if f], key=key)
                assert (pu == best).all()


@pytest.mark.parametrize("r2", [1, 2, 3, 5, 9, 14])
def test_dilate_single_voxel_is_the_lattice_ball(r2):
    occ = np.zeros((15, 15, 15), np.uint8)
    occ[7, 7, 7] = 1
    out = O.dilate(occ, r2)
    z, y, x = np.mgrid[0:15, 0:15, 0:15]
    ball = (x - 7) ** 2 + (y - 7) ** 2 + (z - 7) ** 2 <= r2
    assert (out.astype(bool) == ball).all()


def test_dilate_matches_scipy_binary_dilation():
    """Against scipy's binary dilation with the ball as structuring element
    (an independent library routine), on random scenes with ragged shapes."""
    from scipy import ndimage
    rng = np.random.default_rng(3)
    for shape in [(32, 9, 7), (20, 21, 11), (64, 5, 6)]:
        nx, ny, nz = shape
        occ = (rng.random((nz, ny, nx)) < 0.03).astype(np.uint8)
        for r2 in (0, 1, 2, 4, 6):
            r = int(np.floor(np.sqrt(r2)))
            k = np.arange(-r, r + 1)
            Z, Y, X = np.meshgrid(k, k, k, indexing="ij")
            st = (X * X + Y * Y + Z * Z) <= r2
            want = ndimage.binary_dilation(occ.astype(bool), structure=st)
            assert (O.dilate(occ, r2).astype(bool) == want).all(), (shape, r2)


def test_dilate_identity_monotone_and_composition():
    rng = np.random.default_rng(4)
    occ = (rng.random((10, 12, 32)) < 0.02).astype(np.uint8)
    assert (O.dilate(occ, 0) == occ).all()
    prev = occ
    for r2 in (1, 2, 3, 4, 5, 6, 8, 9):
        cur = O.dilate(occ, r2)
        assert (cur >= prev).all()
        prev = cur
    # the cube of half-width 1 is the ball r2 = 3; dilating twice by it is
    # the cube of half-width 2, which lies between the balls r2 = 4 and 12
    once = O.dilate(occ, 3)
    twice = O.dilate(once, 3)
    assert (twice >= O.dilate(occ, 4)).all() and (twice <= O.dilate(occ, 12)).all()


def _limited_chains(occ_bool, bounds, limits):
    ch = BF.Chains(occ_bool, bounds)
    for k, c in enumerate(limits):
        if c is not None:
            ch.offs[k] = [tuple(int(v) for v in d) for d in _cone_offsets(*bounds[k], (c[:3], c[3], c[4]))]
    return ch


LIMITS = [
    [(0, 0, 1, 0, 1), None, None],            # first segment in the upper half-space
    [(0, 0, 1, 1, 4), (1, 0, 0, 0, 1), None],
    [None, (0, 1, 1, 1, 3), (0, 0, -1, 0, 1)],
]


@pytest.mark.parametrize("scene", range(3))
def test_segment_limits_vs_enumeration(scene):
    """Per-segment direction limits (Step 1 (a) of "The procedure for IK
    solution"): F, V and the reach pose against enumeration of every chain
    whose segments lie in their cones."""
    shape, lengths, n_boxes, seed = TINY[scene]
    rng = np.random.default_rng(700 + seed)
    nx, ny, nz = shape
    root = (nx // 2, ny // 2, 0)
    boxes = _rand_scene(rng, shape, n_boxes, 3, keep=[root])
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    S = len(lengths)
    for lim in LIMITS:
        lim = lim[:S] + [None] * max(0, S - len(lim))
        ch = _limited_chains(BF.occupancy(shape, boxes), bounds, lim)
        F = O.forward(occ, lengths, root, limits=lim)
        targets = [tuple(int(v) for v in rng.integers(0, [nx, ny, nz])) for _ in range(5)]
        poses, found, vs = O.reach_many(occ, lengths, root, targets, want_sets=True, limits=lim)
        for i, t in enumerate(targets):
            Fb, Vb, good = ch.joint_sets(root, [t])
            for k in range(S + 1):
                assert BF.to_set(F[k]) == Fb[k], ("F", k)
                assert BF.to_set(vs[i, k]) == Vb[k], ("V", t, k)
            assert bool(found[i]) == bool(good)
            if good:
                assert tuple(map(tuple, poses[i].tolist())) == ch.lexmin(good)
                assert O.pose_valid(occ, lengths, poses[i], limits=lim)


def test_upper_half_space_closed_form():
    """Segment 1 limited to s_z > 0: F_1 is the unlimited F_1 above the root's
    plane, and a pose whose first segment points down is invalid."""
    shape, lengths = (12, 12, 10), (3, 2, 2)
    rng = np.random.default_rng(5)
    root = (6, 6, 3)
    boxes = _rand_scene(rng, shape, 6, 3, keep=[root])
    occ = O.rasterize(shape, boxes)
    lim = [(0, 0, 1, 0, 1), None, None]
    F = O.forward(occ, lengths, root, limits=lim)
    F0 = O.forward(occ, lengths, root)
    z = np.arange(shape[2])[:, None, None]
    assert (F[1] == (F0[1] * (z > root[2]))).all()
    assert (F[2] <= F0[2]).all() and (F[3] <= F0[3]).all()
    poses, found, _ = O.reach_many(occ, lengths, root, [tuple(int(v) for v in np.argwhere(F0[3])[0][::-1])])
    if found[0] and poses[0][1][2] <= root[2]:
        assert not O.pose_valid(occ, lengths, poses[0], limits=lim)


@pytest.mark.parametrize("seed", range(2))
def test_plan_path_with_limits_vs_enumeration(seed):
    rng = np.random.default_rng(800 + seed)
    shape = (10, 10, 8)
    lengths = (3, 3, 2)
    root = (5, 5, 0)
    lim = [(0, 0, 1, 1, 4), None, (0, 0, -1, 0, 1)]
    boxes = _rand_scene(rng, shape, 5, 2, keep=[root])
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    ch = _limited_chains(BF.occupancy(shape, boxes), bounds, lim)
    free = np.argwhere(occ == 0)[:, ::-1]
    for _ in range(80):
        t = tuple(int(v) for v in free[rng.integers(len(free))])
        poses, found, _ = O.reach_many(occ, lengths, root, [t], limits=lim)
        if found[0]:
            break
    assert found[0]
    W, delta = 6, 1
    p_o, r_o, st = O.plan_path(occ, lengths, poses[0], W, delta=delta, eps2=1, eps2_max=4, limits=lim)
    p_b, r_b = _brute_plan(ch, lengths, poses[0], W, delta, 1, 4)
    assert [tuple(map(tuple, p.tolist())) for p in p_o] == p_b
    assert r_o.tolist() == r_b


def test_backward_sets_vs_enumeration():
    shape, lengths = (8, 7, 6), (3, 2, 2)
    rng = np.random.default_rng(11)
    boxes = _rand_scene(rng, shape, 4, 3)
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    ch = BF.Chains(BF.occupancy(shape, boxes), bounds)
    T = np.zeros(occ.shape, np.uint8)
    t = (4, 3, 2)
    T[t[2], t[1], t[0]] = 1
    B = O.backward(occ, lengths, T)
    S = len(lengths)
    for k in range(S + 1):
        # B_k = voxels p from which segments k+1..S reach t
        want = set()
        for z in range(shape[2]):
            for y in range(shape[1]):
                for x in range(shape[0]):
                    p = (x, y, z)
                    if not ch.free(p):
                        continue
                    for chain in _chains_from(ch, p, k, S):
                        if chain[-1] == t:
                            want.add(p)
                            break
        assert BF.to_set(B[k]) == want, k


def _chains_from(ch, p, k, S):
    if k == S:
        yield (p,)
        return
    for d in ch.offs[k]:
        q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
        if ch.inside(q) and ch.edge(p, q):
            for rest in _chains_from(ch, q, k + 1, S):
                yield (p,) + rest


# --------------------------------------------------------------- closed forms

def test_free_space_closed_forms():
    shape = (24, 22, 20)
    occ = np.zeros((20, 22, 24), np.uint8)
    lengths = (5, 4)
    root, t = (12, 11, 0), (15, 16, 6)
    F = O.forward(occ, lengths, root)
    lo1, hi1 = O.shell_bounds(5)
    lo2, hi2 = O.shell_bounds(4)
    sh1 = BF.shell_offsets(lo1, hi1)
    sh2 = BF.shell_offsets(lo2, hi2)
    inside = lambda p: 0 <= p[0] < 24 and 0 <= p[1] < 22 and 0 <= p[2] < 20
    want_f1 = {tuple(int(v) for v in np.asarray(root) + d) for d in sh1}
    want_f1 = {p for p in want_f1 if inside(p)}
    assert BF.to_set(F[1]) == want_f1
    _, found, vs = O.reach_many(occ, lengths, root, [t], want_sets=True)
    want_v1 = want_f1 & {tuple(int(v) for v in np.asarray(t) - d) for d in sh2}
    assert BF.to_set(vs[0, 1]) == want_v1
    assert bool(found[0]) == bool(want_v1)


def test_one_segment_iff():
    rng = np.random.default_rng(9)
    shape = (16, 16, 16)
    boxes = _rand_scene(rng, shape, 10, 3, keep=[(8, 8, 0)])
    occ = O.rasterize(shape, boxes)
    occb = occ.astype(bool)
    root = (8, 8, 0)
    lo, hi = O.shell_bounds(6)
    targets = [tuple(int(v) for v in rng.integers(0, 16, 3)) for _ in range(60)]
    _, found, _ = O.reach_many(occ, (6,), root, targets)
    for t, f in zip(targets, found):
        d = np.asarray(t) - np.asarray(root)
        ok = lo <= int(d @ d) <= hi and all(not occb[v[2], v[1], v[0]]
                                             for v in BF.supercover(root, t))
        assert bool(f) == ok, t


def test_empty_beyond_reach_and_occupied_endpoints():
    sc = G.c1_scene(0)
    occ = O.rasterize(sc.shape, sc.boxes)
    reach = sum(L + 0.5 for L in sc.lengths)
    far = [t for t in [(0, 0, 31), (31, 31, 31), (0, 31, 31)]
           if sum((a - b) ** 2 for a, b in zip(t, sc.root)) > reach ** 2]
    occd = np.argwhere(occ)[:3][:, ::-1]  # occupied voxels as (x, y, z)
    targets = far + [tuple(int(v) for v in p) for p in occd]
    _, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets)
    assert not found.any()
    # an occupied root: nothing is reachable
    b = np.concatenate([sc.boxes, [[16, 16, 0, 16, 16, 0]]]).astype(np.int32)
    occ2 = O.rasterize(sc.shape, b)
    F = O.forward(occ2, sc.lengths, sc.root)
    assert F.sum() == 0


# ------------------------------------------------- dualities and monotonicity

def test_reverse_arm_duality():
    rng = np.random.default_rng(21)
    shape = (14, 13, 12)
    boxes = _rand_scene(rng, shape, 8, 3)
    occ = O.rasterize(shape, boxes)
    lengths = (4, 3, 5)
    free = np.argwhere(occ == 0)[:, ::-1]
    for trial in range(4):
        r = tuple(int(v) for v in free[rng.integers(len(free))])
        t = tuple(int(v) for v in free[rng.integers(len(free))])
        _, f1, v1 = O.reach_many(occ, lengths, r, [t], want_sets=True)
        _, f2, v2 = O.reach_many(occ, lengths[::-1], t, [r], want_sets=True)
        assert f1[0] == f2[0]
        S = len(lengths)
        for k in range(S + 1):
            assert (v1[0, k] == v2[0, S - k]).all(), (trial, k)


def test_mirror_symmetry():
    rng = np.random.default_rng(22)
    shape = (16, 12, 10)
    boxes = _rand_scene(rng, shape, 8, 3, keep=[(7, 6, 0)])
    occ = O.rasterize(shape, boxes)
    lengths = (4, 4, 3)
    r, t = (7, 6, 0), (10, 8, 5)
    _, _, v1 = O.reach_many(occ, lengths, r, [t], want_sets=True)
    occ_m = occ[:, :, ::-1].copy()
    rm, tm = (shape[0] - 1 - r[0], r[1], r[2]), (shape[0] - 1 - t[0], t[1], t[2])
    _, _, v2 = O.reach_many(occ_m, lengths, rm, [tm], want_sets=True)
    assert (v1[0][..., ::-1] == v2[0]).all()


def test_monotone_in_obstacles():
    rng = np.random.default_rng(23)
    shape = (16, 16, 12)
    root = (8, 8, 0)
    boxes = _rand_scene(rng, shape, 6, 3, keep=[root])
    more = np.concatenate([boxes, _rand_scene(rng, shape, 6, 3, keep=[root])])
    occ_a = O.rasterize(shape, boxes)
    occ_b = O.rasterize(shape, more)
    lengths = (5, 4, 3)
    t = (10, 12, 5)
    Fa = O.forward(occ_a, lengths, root)
    Fb = O.forward(occ_b, lengths, root)
    assert (Fb <= Fa).all()
    _, _, va = O.reach_many(occ_a, lengths, root, [t], want_sets=True)
    _, _, vb = O.reach_many(occ_b, lengths, root, [t], want_sets=True)
    assert (vb <= va).all()


def test_v_subset_of_f_and_pose_invariants_c1():
    for seed in range(3):
        sc = G.c1_scene(seed)
        occ = O.rasterize(sc.shape, sc.boxes)
        targets = G.draw_targets(sc, 3, seed)
        F = O.forward(occ, sc.lengths, sc.root)
        poses, found, vs = O.reach_many(occ, sc.lengths, sc.root, targets, want_sets=True)
        for i, t in enumerate(targets):
            assert (vs[i] <= F).all()
            if not found[i]:
                continue
            p = poses[i]
            assert tuple(p[0]) == sc.root and tuple(p[-1]) == tuple(t)
            assert O.pose_valid(occ, sc.lengths, p)
            for k, L in enumerate(sc.lengths, start=1):
                d = p[k] - p[k - 1]
                assert L * L - L + 1 <= int(d @ d) <= L * L + L
                assert vs[i, k, p[k][2], p[k][1], p[k][0]]


# ----------------------------------------------------------------- guide

def _guide_fraction(lengths, pose, W):
    """Guide points by exact rational arc parameter, rounding half up."""
    lam = sum(lengths)
    C = np.concatenate([[0], np.cumsum(lengths)])
    out = []
    for j in range(W):
        s = Fraction(j * lam, W - 1)
        k = len(lengths)
        for kk in range(1, len(lengths) + 1):
            if C[kk - 1] <= s < C[kk]:
                k = kk
                break
        f = (s - int(C[k - 1])) / lengths[k - 1]
        a, b = pose[k - 1], pose[k]
        out.append(tuple(int(a[i]) + floor(f * int(b[i] - a[i]) + Fraction(1, 2))
                         for i in range(3)))
    return out


def test_guide_against_rational_rule():
    rng = np.random.default_rng(4)
    for _ in range(40):
        S = int(rng.integers(2, 9))
        lengths = [int(v) for v in rng.integers(2, 25, S)]
        pose = np.cumsum(np.concatenate([[rng.integers(0, 50, 3)],
                                         rng.integers(-20, 21, (S, 3))]), axis=0)
        W = int(rng.integers(2, 40))
        g = O.guide(lengths, pose, W)
        assert [tuple(v) for v in g.tolist()] == _guide_fraction(lengths, pose, W)
        assert tuple(g[0]) == tuple(pose[0]) and tuple(g[-1]) == tuple(pose[-1])


def test_guide_straight_arm():
    lengths = [4, 3, 5]
    pose = np.array([[0, 0, 0], [4, 0, 0], [7, 0, 0], [12, 0, 0]])
    g = O.guide(lengths, pose, 7)  # spacing 2 along x
    assert g[:, 0].tolist() == [0, 2, 4, 6, 8, 10, 12]
    assert (g[:, 1:] == 0).all()


# ---------------------------------------------------------------- path (tiny)

def _ball_chains(ch, root, ref, delta, targets):
    """All valid chains with joint k within delta of ref[k], ending in targets."""
    out = []
    S = ch.S
    d2 = delta * delta

    def rec(chain, k):
        if k > S:
            if chain[-1] in targets:
                out.append(tuple(chain))
            return
        p = chain[-1]
        for d in ch.offs[k - 1]:
            q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
            if not ch.inside(q):
                continue
            if sum((q[i] - ref[k][i]) ** 2 for i in range(3)) > d2:
                continue
            if ch.edge(p, q):
                chain.append(q)
                rec(chain, k + 1)
                chain.pop()

    rec([root], 1)
    return out


def _brute_plan(ch, lengths, reach, W, delta, eps2, eps2_max, guide=None):
    """The planning rule with each smooth step solved by enumeration (guide:
    the guide points, else those of the reach pose)."""
    S = len(lengths)
    g = _guide_fraction(lengths, reach, W) if guide is None else guide
    poses = [None] * W
    relax = [[0, 0] for _ in range(W)]
    poses[W - 1] = tuple(map(tuple, np.asarray(reach).tolist()))
    root = poses[W - 1][0]
    diag2 = (ch.nx - 1) ** 2 + (ch.ny - 1) ** 2 + (ch.nz - 1) ** 2
    for j in range(W - 2, -1, -1):
        T, used = set(), -1
        for e2 in range(eps2, max(eps2, eps2_max) + 1):
            T = {(x, y, z) for z in range(ch.nz) for y in range(ch.ny) for x in range(ch.nx)
                 if (x - g[j][0]) ** 2 + (y - g[j][1]) ** 2 + (z - g[j][2]) ** 2 <= e2
                 and ch.free((x, y, z))}
            if T:
                used = e2
                break
        relax[j][1] = used
        ref = poses[j + 1]
        m = 0
        while True:
            d = delta + m
            good = _ball_chains(ch, root, ref, d, T)
            if good:
                poses[j] = ch.lexmin(good)
                relax[j][0] = m
                break
            if d * d >= diag2:
                poses[j] = ref
                relax[j][0] = -1
                break
            m += 1
    return poses, relax


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_path_vs_enumeration(seed):
    rng = np.random.default_rng(300 + seed)
    shape = (10, 10, 8)
    lengths = (3, 3, 2)
    root = (5, 5, 0)
    boxes = _rand_scene(rng, shape, 5, 2, keep=[root])
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    ch = BF.Chains(BF.occupancy(shape, boxes), bounds)
    free = np.argwhere(occ == 0)[:, ::-1]
    # a reachable target
    for _ in range(50):
        t = tuple(int(v) for v in free[rng.integers(len(free))])
        poses, found, _ = O.reach_many(occ, lengths, root, [t])
        if found[0]:
            break
    assert found[0]
    reach = poses[0]
    W, delta = 6, 1
    p_o, r_o, st = O.plan_path(occ, lengths, reach, W, delta=delta, eps2=1, eps2_max=4)
    p_b, r_b = _brute_plan(ch, lengths, reach, W, delta, 1, 4)
    assert [tuple(map(tuple, p.tolist())) for p in p_o] == p_b
    assert r_o.tolist() == r_b
    want = (O.PATH_BROKEN if any(r[0] < 0 for r in r_b) else
            O.PATH_RELAXED if any(r[0] > 0 or (r[1] != 1) for r in r_b[:-1]) else O.PATH_OK)
    assert st == want


def test_plan_path_invariants_c1():
    sc = G.c1_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 2, 1)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets)
    for i in range(len(targets)):
        if not found[i]:
            continue
        W = 8
        path, relax, st = O.plan_path(occ, sc.lengths, poses[i], W, delta=3)
        g = O.guide(sc.lengths, poses[i], W)
        assert (path[-1] == poses[i]).all()
        for j in range(W):
            assert O.pose_valid(occ, sc.lengths, path[j])
            assert tuple(path[j][0]) == sc.root
            if j < W - 1 and relax[j][0] >= 0:
                e = path[j][-1] - g[j]
                assert int(e @ e) <= relax[j][1]
                step = path[j] - path[j + 1]
                d = 3 + relax[j][0]
                assert (np.sum(step * step, axis=1) <= d * d).all()


# ------------------------------------------------------------- short reaches

def _brute_short(shape, boxes, lengths, reach, kmax):
    """The first virtual arm (L_1 .. L_{k-1}, l) in the order k, then l, whose
    chains from the root reach the target, by enumeration; (k, l, lengths,
    lexicographically smallest chain) or None."""
    occb = BF.occupancy(shape, boxes)
    root = tuple(int(v) for v in reach[0])
    t = tuple(int(v) for v in reach[-1])
    for k in range(1, min(kmax, len(lengths)) + 1):
        for l in range(1, lengths[k - 1] + 1):
            vl = list(lengths[:k])
            vl[-1] = l
            ch = BF.Chains(occb, [O.shell_bounds(v) for v in vl])
            _, _, good = ch.joint_sets(root, [t])
            if good:
                return k, l, vl, ch.lexmin(good)
    return None


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_plan_short_vs_enumeration(seed):
    rng = np.random.default_rng(1200 + seed)
    shape = (10, 10, 8)
    lengths = (3, 3, 2)
    root = (5, 5, 0)
    boxes = _rand_scene(rng, shape, 5, 2, keep=[root])
    occ = O.rasterize(shape, boxes)
    ch = BF.Chains(BF.occupancy(shape, boxes), [O.shell_bounds(L) for L in lengths])
    free = np.argwhere(occ == 0)[:, ::-1]
    n_short = 0
    for _ in range(40):
        t = tuple(int(v) for v in free[rng.integers(len(free))])
        poses, found, _ = O.reach_many(occ, lengths, root, [t])
        if not found[0]:
            continue
        reach = poses[0]
        W, delta = 5, 1
        p_o, r_o, st, kl, vpose = O.plan_short(occ, lengths, reach, W, delta=delta, eps2=1, eps2_max=4)
        want = _brute_short(shape, boxes, lengths, reach, 2)
        if want is None:
            assert kl == (0, 0) and vpose is None
            guide = None
        else:
            k, l, vl, vchain = want
            assert kl == (k, l)
            assert [tuple(v) for v in vpose.tolist()] == list(vchain)
            guide = _guide_fraction(vl, np.array(vchain), W)
            n_short += 1
        p_b, r_b = _brute_plan(ch, lengths, reach, W, delta, 1, 4, guide=guide)
        assert [tuple(map(tuple, p.tolist())) for p in p_o] == p_b
        assert r_o.tolist() == r_b
        if n_short >= 2:
            break
    assert n_short >= 1


def test_plan_short_falls_back_to_the_reach_polyline():
    # the root itself as target: no virtual arm of length >= 1 ends there
    sc = G.c1_scene(0)
    occ = O.rasterize(sc.shape, sc.boxes)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, [sc.root])
    if not found[0]:
        pytest.skip("no pose ends at the root in this scene")
    p_s, r_s, st_s, kl, vpose = O.plan_short(occ, sc.lengths, poses[0], 6)
    p_p, r_p, st_p = O.plan_path(occ, sc.lengths, poses[0], 6)
    assert kl == (0, 0) and vpose is None
    assert (p_s == p_p).all() and (r_s == r_p).all() and st_s == st_p


# ------------------------------------------ follower path (the paper's form)

def _guide_follow_fraction(pose, F, n):
    """n guide points per segment up to joint F, exact, rounding half up."""
    out = []
    for k in range(1, F + 1):
        a, b = pose[k - 1], pose[k]
        for i in range(n):
            out.append(tuple(int(a[c]) + floor(Fraction(i, n) * int(b[c] - a[c]) + Fraction(1, 2))
                             for c in range(3)))
    out.append(tuple(int(v) for v in pose[F]))
    return out


def _fold_target(lengths, pose, F, n, j):
    """The point L_S further along the reach polyline than guide point j
    (nominal arc lengths), as exact fractions."""
    S = len(lengths)
    C = [0]
    for L in lengths:
        C.append(C[-1] + L)
    k, i = j // n + 1, j % n
    if k > F:
        k, i = F, n
    s = C[k - 1] + Fraction(i * lengths[k - 1], n) + lengths[S - 1]
    kk = S
    for q in range(1, S + 1):
        if C[q - 1] <= s < C[q]:
            kk = q
            break
    f = (s - C[kk - 1]) / lengths[kk - 1]
    a, b = pose[kk - 1], pose[kk]
    return tuple(int(a[c]) + f * int(b[c] - a[c]) for c in range(3))


def _radius_chains(ch, root, ref, r2, targets):
    """All valid chains with joint k within sqrt(r2[k]) of ref[k] (r2[k] < 0:
    anywhere), ending in targets."""
    out = []

    def rec(chain, k):
        if k > ch.S:
            if chain[-1] in targets:
                out.append(tuple(chain))
            return
        p = chain[-1]
        for d in ch.offs[k - 1]:
            q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
            if not ch.inside(q):
                continue
            if r2[k] >= 0 and sum((q[i] - ref[k][i]) ** 2 for i in range(3)) > r2[k]:
                continue
            if ch.edge(p, q):
                chain.append(q)
                rec(chain, k + 1)
                chain.pop()

    rec([root], 1)
    return out


def _brute_follow(ch, chF, lengths, reach, n, fold, rad, eps2, eps2_max):
    """The follower rule with each smooth step solved by enumeration and the
    folded segment by a scan of its shell."""
    S = len(lengths)
    F = S - (1 if fold else 0)
    W = F * n + 1
    g = _guide_follow_fraction(reach, F, n)
    rt = tuple(tuple(int(v) for v in p) for p in np.asarray(reach).tolist())
    root = rt[0]
    tp = [None] * W
    relax = [[0, 0] for _ in range(W)]
    tp[W - 1] = rt[:F + 1]
    diag2 = (ch.nx - 1) ** 2 + (ch.ny - 1) ** 2 + (ch.nz - 1) ** 2
    for j in range(W - 2, -1, -1):
        T, used = set(), -1
        for e2 in range(eps2, max(eps2, eps2_max) + 1):
            T = {(x, y, z) for z in range(ch.nz) for y in range(ch.ny) for x in range(ch.nx)
                 if (x - g[j][0]) ** 2 + (y - g[j][1]) ** 2 + (z - g[j][2]) ** 2 <= e2
                 and ch.free((x, y, z))}
            if T:
                used = e2
                break
        relax[j][1] = used
        ref = tp[j + 1]
        m = 0
        while True:
            r2 = [None] + [-1 if r < 0 else (r + m) ** 2 for r in rad]
            good = _radius_chains(chF, root, ref, r2, T)
            if good:
                tp[j] = chF.lexmin(good)
                relax[j][0] = m
                break
            if all(r < 0 or (r + m) ** 2 >= diag2 for r in rad):
                tp[j] = ref
                relax[j][0] = -1
                break
            m += 1
    full = []
    for j in range(W):
        pose = list(tp[j])
        if fold:
            a = _fold_target(lengths, reach, F, n, j)
            f = pose[F]
            best = None
            for d in ch.offs[S - 1]:
                q = (f[0] + d[0], f[1] + d[1], f[2] + d[2])
                if not ch.inside(q) or not ch.edge(f, q):
                    continue
                key = (sum((q[c] - a[c]) ** 2 for c in range(3)), ch.index(q))
                if best is None or key < best[0]:
                    best = (key, q)
            if best is None:
                pose.append(f)
                relax[j][0] = -1
            else:
                pose.append(best[1])
        full.append(tuple(pose))
    return full, relax


def test_guide_follow_straight_arm():
    # segments along x of lengths 4, 3, 5: two points per segment up to joint 2
    lengths = [4, 3, 5]
    pose = np.array([[0, 0, 0], [4, 0, 0], [7, 0, 0], [12, 0, 0]])
    assert _guide_follow_fraction(pose, 2, 2) == [(0, 0, 0), (2, 0, 0), (4, 0, 0), (6, 0, 0), (7, 0, 0)]
    # the fold target of the last waypoint is the end effector; of the first,
    # the point 5 voxels along the polyline from the root
    assert _fold_target(lengths, pose, 2, 2, 4) == (12, 0, 0)
    assert _fold_target(lengths, pose, 2, 2, 0) == (5, 0, 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("fold", [True, False])
def test_plan_path_follow_vs_enumeration(seed, fold):
    rng = np.random.default_rng(900 + seed)
    shape = (10, 10, 8)
    lengths = (3, 3, 2, 2)
    root = (5, 5, 0)
    boxes = _rand_scene(rng, shape, 5, 2, keep=[root])
    occ = O.rasterize(shape, boxes)
    bounds = [O.shell_bounds(L) for L in lengths]
    F = len(lengths) - (1 if fold else 0)
    ch = BF.Chains(BF.occupancy(shape, boxes), bounds)
    chF = BF.Chains(BF.occupancy(shape, boxes), bounds[:F])
    free = np.argwhere(occ == 0)[:, ::-1]
    for _ in range(50):
        t = tuple(int(v) for v in free[rng.integers(len(free))])
        poses, found, _ = O.reach_many(occ, lengths, root, [t])
        if found[0]:
            break
    assert found[0]
    reach = poses[0]
    n = 2
    rad = [1, 2] + [-1] * (F - 2)
    p_o, r_o, st = O.plan_path_follow(occ, lengths, reach, n, fold, rad, eps2=1, eps2_max=4)
    p_b, r_b = _brute_follow(ch, chF, lengths, reach, n, fold, rad, 1, 4)
    assert [tuple(map(tuple, p.tolist())) for p in p_o] == p_b
    assert r_o.tolist() == r_b
    want = (O.PATH_BROKEN if any(r[0] < 0 for r in r_b) else
            O.PATH_RELAXED if any(r[0] > 0 or (r[1] != 1) for r in r_b[:-1]) else O.PATH_OK)
    assert st == want
    assert (p_o[-1] == reach).all()


def test_plan_path_follow_invariants_c1():
    sc = G.c1_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 3, 2)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets)
    S = len(sc.lengths)
    n, rad = 4, [2, 3, -1]
    ch = BF.Chains(BF.occupancy(sc.shape, sc.boxes), [O.shell_bounds(L) for L in sc.lengths])
    for i in np.nonzero(found)[0]:
        path, relax, st = O.plan_path_follow(occ, sc.lengths, poses[i], n, True, rad)
        g = _guide_follow_fraction(poses[i], S - 1, n)
        assert len(path) == (S - 1) * n + 1 and (path[-1] == poses[i]).all()
        for j in range(len(path)):
            if relax[j][0] < 0:
                continue
            assert O.pose_valid(occ, sc.lengths, path[j])
            e = path[j][S - 1] - np.array(g[j])
            assert int(e @ e) <= max(relax[j][1], 0)
            if j < len(path) - 1:
                step = path[j] - path[j + 1]
                for k in (1, 2):
                    d = rad[k - 1] + relax[j][0]
                    assert int(step[k] @ step[k]) <= d * d
            # the folded end: nearest free shell end to the fold target
            a = _fold_target(sc.lengths, poses[i], S - 1, n, j)
            f = tuple(int(v) for v in path[j][S - 1])
            best = None
            for d in ch.offs[S - 1]:
                q = (f[0] + d[0], f[1] + d[1], f[2] + d[2])
                if ch.inside(q) and ch.edge(f, q):
                    key = (sum((q[c] - a[c]) ** 2 for c in range(3)), ch.index(q))
                    best = key if best is None or key < best else best
            assert best is not None and ch.index(tuple(int(v) for v in path[j][S])) == best[1]


def test_plan_path_follow_rejects_invalid_reach():
    sc = G.c1_scene(1)
    occ = O.rasterize(sc.shape, sc.boxes)
    bad = np.zeros((len(sc.lengths) + 1, 3), np.int32)
    path, relax, st = O.plan_path_follow(occ, sc.lengths, bad, 2, True, [2, 3, -1])
    assert path is None and st == O.PATH_UNREACHABLE


# -------------------------------------------------------------------- replan

def test_replan_keeps_valid_path_and_fixes_cut():
    sc = G.c1_scene(2)
    occ = O.rasterize(sc.shape, sc.boxes)
    targets = G.draw_targets(sc, 4, 2)
    poses, found, _ = O.reach_many(occ, sc.lengths, sc.root, targets)
    i = int(np.argmax(found))
    W = 8
    path, relax, st = O.plan_path(occ, sc.lengths, poses[i], W)
    kept, _, st2 = O.replan(occ, sc.lengths, path, 2)
    assert st2 == O.PATH_KEPT and (kept == path).all()
    # cut the path: put a small box on a mid-path joint of a later pose
    j = W - 3
    v = path[j][2]
    box = np.array([[v[0], v[1], v[2], v[0], v[1], v[2]]], np.int32)
    occ2 = O.rasterize(sc.shape, np.concatenate([sc.boxes, box]))
    assert not O.pose_valid(occ2, sc.lengths, path[j])
    new, relax2, st3 = O.replan(occ2, sc.lengths, path, 2)
    assert st3 != O.PATH_KEPT
    assert (new[:3] == path[:3]).all()
    if st3 in (O.PATH_OK, O.PATH_RELAXED):
        for jj in range(3, W):
            assert O.pose_valid(occ2, sc.lengths, new[jj])
            step = new[jj] - new[jj - 1]
            d = 3 + relax2[jj][0]
            assert (np.sum(step * step, axis=1) <= d * d).all()


def _brute_valid(ch, pose):
    """A pose is valid when every segment is a shell offset of its length
    with an obstacle-free closed supercover inside the grid (enumeration's
    own edge test)."""
    for k in range(1, len(pose)):
        p, q = tuple(pose[k - 1]), tuple(pose[k])
        d2 = sum((q[i] - p[i]) ** 2 for i in range(3))
        lo, hi = ch.bounds[k - 1]
        if not (lo <= d2 <= hi and ch.edge(p, q)):
            return False
    return True


def _brute_replan(ch, lengths, old, c, delta, eps2, eps2_max):
    """The replan rule (section "Dynamic Obstacles") by enumeration: keep the
    path when every pose after c is still valid; else keep the reach pose if
    valid, or take among ALL valid chains from the root to the old target the
    one whose joints are nearest the old reach pose's, compared joint by joint
    from the root (squared distance, then linear index) -- a lexicographic
    minimum over the enumerated chains, not a greedy walk over sets; then
    chain poses c+1 .. W-1 forward from pose c, each the smallest chain inside
    the balls around the previous pose, with T_{W-1} the reach pose's end."""
    S, W = len(lengths), len(old)
    old = [tuple(tuple(int(v) for v in p) for p in pose) for pose in old]
    relax = [[0, 0] for _ in range(W)]
    if all(_brute_valid(ch, old[j]) for j in range(c + 1, W)):
        return old, relax, O.PATH_KEPT, None
    root = old[0][0]
    reach = old[W - 1]
    resolved = None
    if not _brute_valid(ch, reach):
        _, _, good = ch.joint_sets(root, [old[W - 1][S]])
        if not good:
            poses = old[:c + 1] + [old[c]] * (W - c - 1)
            for j in range(c + 1, W):
                relax[j][0] = -1
            return poses, relax, O.PATH_UNREACHABLE, None

        def key(chain):
            return tuple(v for k in range(1, S + 1)
                         for v in (sum((chain[k][i] - old[W - 1][k][i]) ** 2 for i in range(3)),
                                   ch.index(chain[k])))
        reach = min(good, key=key)
        resolved = (reach, ch.lexmin(good))
    g = _guide_fraction(lengths, np.asarray(reach), W)
    poses = list(old[:c + 1]) + [None] * (W - c - 1)
    diag2 = (ch.nx - 1) ** 2 + (ch.ny - 1) ** 2 + (ch.nz - 1) ** 2
    relaxed = broken = False
    for j in range(c + 1, W):
        if j == W - 1:
            T, used = {reach[S]}, 0
        else:
            T, used = set(), -1
            for e2 in range(eps2, max(eps2, eps2_max) + 1):
                T = {(x, y, z) for z in range(ch.nz) for y in range(ch.ny) for x in range(ch.nx)
                     if (x - g[j][0]) ** 2 + (y - g[j][1]) ** 2 + (z - g[j][2]) ** 2 <= e2
                     and ch.free((x, y, z))}
                if T:
                    used = e2
                    break
            relaxed |= used != eps2
        relax[j][1] = used
        ref = poses[j - 1]
        m = 0
        while True:
            d = delta + m
            good = _ball_chains(ch, root, ref, d, T)
            if good:
                poses[j] = ch.lexmin(good)
                relax[j][0] = m
                relaxed |= m > 0
                break
            if d * d >= diag2:
                poses[j] = ref
                relax[j][0] = -1
                broken = True
                break
            m += 1
    st = O.PATH_BROKEN if broken else (O.PATH_RELAXED if relaxed else O.PATH_OK)
    return poses, relax, st, resolved


def _replan_cases():
    """Tiny scenes, each with a planned path and the cuts that exercise every
    branch of the replan rule: nothing cut; a later pose cut but the reach
    pose kept; a joint of the reach pose (or a voxel of its segment) cut, so
    that the reach pose is re-solved; the target itself occupied."""
    cases = []
    for seed in range(4):
        rng = np.random.default_rng(1200 + seed)
        shape = (10, 10, 8)
        lengths = (3, 3, 2)
        root = (5, 5, 0)
        boxes = _rand_scene(rng, shape, 4, 2, keep=[root])
        occ = O.rasterize(shape, boxes)
        free = np.argwhere(occ == 0)[:, ::-1]
        for _ in range(80):
            t = tuple(int(v) for v in free[rng.integers(len(free))])
            poses, found, _ = O.reach_many(occ, lengths, root, [t])
            if found[0]:
                break
        assert found[0]
        W = 6
        path, _, _ = O.plan_path(occ, lengths, poses[0], W, delta=1, eps2=1, eps2_max=4)
        reach = path[W - 1]
        cuts = [("none", None)]
        j = W - 3
        cuts.append(("mid pose", tuple(int(v) for v in path[j][2])))
        cuts.append(("reach joint 1", tuple(int(v) for v in reach[1])))
        cuts.append(("reach joint 2", tuple(int(v) for v in reach[2])))
        r2, r3 = (tuple(int(v) for v in reach[k]) for k in (2, 3))
        sc_mid = [tuple(int(v) for v in p) for p in BF.supercover(r2, r3) if tuple(p) not in (r2, r3)]
        if sc_mid:
            cuts.append(("reach segment 3", sc_mid[len(sc_mid) // 2]))
        cuts.append(("target", tuple(int(v) for v in reach[3])))
        for name, v in cuts:
            if v is not None and v == root:
                continue
            b = boxes if v is None else np.concatenate(
                [boxes, np.asarray([[*v, *v]], np.int32)])
            for c in (1, 2):
                cases.append((f"seed {seed}, cut {name}, c={c}", shape, lengths, b, path, c))
    return cases


def _replan_mismatches(cases, delta=1, eps2=1, eps2_max=4, first=False):
    bad, counts, differs = [], {}, 0
    for name, shape, lengths, boxes, path, c in cases:
        occ = O.rasterize(shape, boxes)
        ch = BF.Chains(BF.occupancy(shape, boxes), [O.shell_bounds(L) for L in lengths])
        p_o, r_o, st = O.replan(occ, lengths, path, c, delta=delta, eps2=eps2, eps2_max=eps2_max)
        p_b, r_b, st_b, resolved = _brute_replan(ch, lengths, path, c, delta, eps2, eps2_max)
        counts[st_b] = counts.get(st_b, 0) + 1
        if resolved is not None and resolved[0] != resolved[1]:
            differs += 1
        same = (st == st_b and r_o.tolist() == r_b
                and [tuple(map(tuple, p.tolist())) for p in p_o] == [tuple(p) for p in p_b])
        if not same:
            bad.append(name)
            if first:
                break
    return bad, counts, differs


def test_replan_vs_enumeration():
    """orc_replan against enumeration on every branch: kept, forward chain
    from pose c with the reach pose kept, the reach pose re-solved (its
    nearest-joint rule checked as a lexicographic minimum over all valid
    chains), and an unreachable target."""
    bad, counts, differs = _replan_mismatches(_replan_cases())
    assert not bad, bad
    # every branch ran, and the re-solve's nearest rule picked a chain other
    # than the plain minimum-index one at least once (so it is discriminated)
    assert counts.get(O.PATH_KEPT, 0) > 0 and counts.get(O.PATH_UNREACHABLE, 0) > 0
    assert counts.get(O.PATH_OK, 0) + counts.get(O.PATH_RELAXED, 0) > 0
    assert differs > 0, counts


# A mistake planted in a copy of the oracle source must fail the replan pin.
_PLANTS = {
    "nearest tie-break by largest index": ("(dd == best_d && qi < best)", "(dd == best_d && qi > best)"),
    "reach re-solve by index only": ("if (best < 0 || dd < best_d ||", "if (best < 0 || false ||"),
    "chain from c + 1": ("int m = smooth_ladder(P, V, poses[j - 1],",
                         "int m = smooth_ladder(P, V, poses[std::max(j - 2, 0)],"),
    "ball target at the last waypoint": ("    if (j == W - 1) {\n      T.assign(P.g.nvox(), 0);\n"
                                         "      T[P.g.index(reach[S].x",
                                         "    if (j == W) {\n      T.assign(P.g.nvox(), 0);\n"
                                         "      T[P.g.index(reach[S].x"),
}


def _oracle_variant(tmp_path, old, new):
    """Build a copy of the oracle with one substitution inside orc_replan."""
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(O.__file__), "ik_oracle.cpp")).read()
    a = src.index("int orc_replan(")
    b = src.index("\n}\n", a)
    body = src[a:b]
    assert body.count(old) == 1, old
    path = tmp_path / "ik_oracle_planted.cpp"
    path.write_text(src[:a] + body.replace(old, new) + src[b:])
    lib = tmp_path / "libik_oracle_planted.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", str(path),
                           "-o", str(lib)])
    return ctypes.CDLL(str(lib))


@pytest.mark.parametrize("plant", sorted(_PLANTS))
def test_planted_mistakes_fail_replan_pin(tmp_path, plant):
    cases = _replan_cases()
    lib = _oracle_variant(tmp_path, *_PLANTS[plant])
    O._load()
    saved = O._lib
    O._lib = lib
    try:
        bad, _, _ = _replan_mismatches(cases, first=True)
    finally:
        O._lib = saved
    assert bad, plant


def test_count_pairs_vs_numpy_shift():
    """orc_count_pairs (the word-pair count of one propagation, section
    "Implementation Performance" cost model restated for bitsets) against a
    numpy formulation: shift the voxel set by each offset, pack 32 voxels of
    a row per word, count the non-zero words; supercover sizes from the
    Chebyshev-distance supercover."""
    rng = np.random.default_rng(77)
    nx, ny, nz = 64, 7, 6
    for L, dens in ((2, 0.02), (3, 0.005), (3, 0.0)):
        X = (rng.random((nz, ny, nx)) < dens).astype(np.uint8)
        if dens > 0:
            X[3, 3, 40] = 1
        lo2, hi2 = O.shell_bounds(L)
        pairs, terms = O.count_pairs(lo2, hi2, X)
        bp = bt = 0
        pad = 4
        Xp = np.zeros((nz + 2 * pad, ny + 2 * pad, nx + 2 * pad), bool)
        Xp[pad:pad + nz, pad:pad + ny, pad:pad + nx] = X.astype(bool)
        for d in BF.shell_offsets(lo2, hi2):
            dx, dy, dz = (int(v) for v in d)
            sh = Xp[pad + dz:pad + dz + nz, pad + dy:pad + dy + ny, pad + dx:pad + dx + nx]
            n = int(sh.reshape(nz, ny, nx // 32, 32).any(axis=3).sum())
            bp += n
            bt += n * len(BF.supercover_from_origin((dx, dy, dz)))
        assert (pairs, terms) == (bp, bt), L
        if dens == 0.0:
            assert pairs == 0


# ---------------------------------------------------------------- generators

def test_splitmix64_published_outputs():
    # splitmix64 from state 0: published first outputs of the generator
    r = G.SplitMix64(0, 0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lemire_uniform_and_range():
    r = G.SplitMix64(5, 1)
    xs = [r.below(7) for _ in range(7000)]
    assert min(xs) == 0 and max(xs) == 6
    counts = np.bincount(xs, minlength=7)
    assert (np.abs(counts - 1000) < 150).all()


def test_scene_shapes():
    sc = G.c2_scene(1)
    assert sc.boxes.shape == (200, 6) and sc.shape == (128, 128, 128)
    assert not sc.point_occupied(sc.root)
    sides = sc.boxes[:, 3:] - sc.boxes[:, :3] + 1
    assert sides.min() >= 1 and sides.max() <= 24
    t = G.draw_targets(sc, 16, 1)
    reach = sum(sc.lengths)
    for p in t:
        assert not sc.point_occupied(tuple(p))
        assert int(((p - np.asarray(sc.root)) ** 2).sum()) <= reach * reach


def _brute_between(ch, chv, lengths, vlengths, start, target, W, delta, eps2, eps2_max):
    """Path between arbitrary poses by enumeration: the virtual arm's
    lexicographically smallest chain from the start's end effector to the
    target, guide points by the rational rule, then each pose the smallest
    chain inside the balls around the previous pose."""
    S = len(lengths)
    vroot = tuple(int(v) for v in start[S])
    _, _, vgood = chv.joint_sets(vroot, [target])
    if not vgood:
        return None
    vpose = chv.lexmin(vgood)
    g = _guide_fraction(vlengths, np.asarray(vpose), W)
    poses = [tuple(map(tuple, np.asarray(start).tolist()))] + [None] * (W - 1)
    relax = [[0, 0] for _ in range(W)]
    root = poses[0][0]
    diag2 = (ch.nx - 1) ** 2 + (ch.ny - 1) ** 2 + (ch.nz - 1) ** 2
    for j in range(1, W):
        if j == W - 1:
            T, used = {tuple(target)}, 0
        else:
            T, used = set(), -1
            for e2 in range(eps2, max(eps2, eps2_max) + 1):
                T = {(x, y, z) for z in range(ch.nz) for y in range(ch.ny) for x in range(ch.nx)
                     if (x - g[j][0]) ** 2 + (y - g[j][1]) ** 2 + (z - g[j][2]) ** 2 <= e2
                     and ch.free((x, y, z))}
                if T:
                    used = e2
                    break
        relax[j][1] = used
        ref = poses[j - 1]
        m = 0
        while True:
            d = delta + m
            good = _ball_chains(ch, root, ref, d, T)
            if good:
                poses[j] = ch.lexmin(good)
                relax[j][0] = m
                break
            if d * d >= diag2:
                poses[j] = ref
                relax[j][0] = -1
                break
            m += 1
    return poses, relax, vpose


@pytest.mark.parametrize("seed", range(3))
def test_plan_between_vs_enumeration(seed):
    """Path between arbitrary poses (section "Path between Arbitrary Poses")
    against enumeration: the virtual arm's pose, the guide, every pose and
    relaxation record."""
    rng = np.random.default_rng(900 + seed)
    shape = (10, 10, 8)
    lengths, vlengths = (3, 3, 2), (2, 2)
    root = (5, 5, 0)
    boxes = _rand_scene(rng, shape, 4, 2, keep=[root])
    occ = O.rasterize(shape, boxes)
    ch = BF.Chains(BF.occupancy(shape, boxes), [O.shell_bounds(L) for L in lengths])
    chv = BF.Chains(BF.occupancy(shape, boxes), [O.shell_bounds(L) for L in vlengths])
    free = np.argwhere(occ == 0)[:, ::-1]
    # a valid start pose: the reach pose of some target
    for _ in range(50):
        t0 = tuple(int(v) for v in free[rng.integers(len(free))])
        p0, f0, _ = O.reach_many(occ, lengths, root, [t0])
        if f0[0]:
            break
    assert f0[0]
    start = p0[0]
    W, delta = 5, 1
    checked = 0
    for _ in range(12):
        target = tuple(int(v) for v in free[rng.integers(len(free))])
        poses, relax, st, vpose = O.plan_between(occ, lengths, start, vlengths, target, W,
                                                 delta=delta, eps2=1, eps2_max=4)
        want = _brute_between(ch, chv, lengths, vlengths, start, target, W, delta, 1, 4)
        if want is None:
            assert st == O.PATH_UNREACHABLE
            assert all((p == start).all() for p in poses)
            continue
        checked += 1
        p_b, r_b, v_b = want
        assert tuple(map(tuple, vpose.tolist())) == v_b
        assert [tuple(map(tuple, p.tolist())) for p in poses] == p_b
        assert relax.tolist() == r_b
        assert (poses[0] == start).all()
    assert checked > 0


def test_plan_between_invalid_start():
    shape, lengths = (10, 10, 8), (3, 3, 2)
    occ = np.zeros((8, 10, 10), np.uint8)
    bad = np.array([[5, 5, 0], [5, 5, 1], [5, 5, 4], [5, 5, 6]], np.int32)  # |s_1| = 1: not a shell offset
    poses, relax, st, _ = O.plan_between(occ, lengths, bad, (2, 2), (3, 3, 3), 4)
    assert st == O.PATH_UNREACHABLE and (relax[1:, 0] == -1).all()
    assert all((p == bad).all() for p in poses)
