"""CPU checks of the CUDA library: it loads, exports every symbol its header
declares, and its host-built tables (shell offsets, incremental supercover)
agree with the oracle's independent constructions.  No compute call needs a
GPU here."""
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "ik.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"IK_API\s+[\w\s\*]+?\b(ik_\w+)\s*\(", text)))


def test_header_symbols_exported(ik):
    declared = _declared_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(ik._lib, name), name
    assert set(declared) == set(ik.EXPORTED)


@pytest.mark.parametrize("L", list(range(1, 25)) + [40, 64, 100])
def test_shell_tables_match_oracle(ik, L):
    (lo, hi), off = ik.ik_shell_offsets(L, 0.5)
    assert (lo, hi) == O.shell_bounds(L, 0.5)
    assert (off == O.shell(lo, hi)).all()


def test_shell_bounds_other_tolerances(ik):
    for tol in (0.0, 0.25, 0.3, 0.75, 0.9):
        for L in (1, 2, 5, 11):
            (lo, hi), _ = ik.ik_shell_offsets(L, tol)
            assert (lo, hi) == O.shell_bounds(L, float(np.float32(tol))), (L, tol)


def test_supercover_traversal_matches_slab_test_every_offset(ik):
    n = 0
    for L in range(1, 25):
        lo, hi = O.shell_bounds(L)
        for d in O.shell(lo, hi):
            a = ik.ik_supercover_offsets(d)
            b = O.supercover((0, 0, 0), d)
            assert a.shape == b.shape and (a == b).all(), (L, d)
            n += 1
    assert n == sum(len(O.shell(*O.shell_bounds(L))) for L in range(1, 25))


def test_supercover_worked_examples(ik):
    got = {tuple(v) for v in ik.ik_supercover_offsets([1, 1, 0]).tolist()}
    assert got == {(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0)}
    assert len(ik.ik_supercover_offsets([1, 1, 1])) == 8
    assert len(ik.ik_supercover_offsets([2, 1, 0])) == 4


def test_bit_layout_roundtrip(ik):
    rng = np.random.default_rng(0)
    m = rng.random((5, 7, 64)) < 0.3
    w = ik.pack_bits(m)
    assert w.dtype == np.uint32 and w.size == 5 * 7 * 2
    # voxel (x, y, z) is bit x % 32 of word (z*ny + y)*(nx/32) + x // 32
    x, y, z = 37, 4, 3
    assert bool((w[(z * 7 + y) * 2 + x // 32] >> (x % 32)) & 1) == bool(m[z, y, x])
    assert (ik.unpack_bits(w, (64, 7, 5))[0] == m).all()


def test_argument_errors_without_gpu(ik):
    with pytest.raises(ik.IkError):
        ik.ik_shell_offsets(0)
    with pytest.raises(ik.IkError):
        ik.ik_supercover_offsets([300, 0, 0])
    assert ik._lib.ik_strerror(-1) == b"invalid argument"


@pytest.mark.parametrize("L", list(range(1, 25)) + [31])
def test_row_lane_table_covers_the_shell_once_in_run_order(ik, L):
    """The row-lane propagation's table (ik_row_table): every offset of the
    shell exactly once; each entry decodes to its offset's dy and shift and
    names its device (edge-mask row) index; the (dz, sign, dy) runs hold
    exactly the offsets of that plane, sign and row, ordered by dx."""
    R, offs, tabr, rowsr = ik.ik_row_table(L)
    (lo2, hi2), shell = ik.ik_shell_offsets(L)
    assert sorted(map(tuple, offs)) == sorted(map(tuple, shell))
    assert R == np.abs(shell).max()
    n = len(offs)
    e = (tabr.astype(np.int64) & 0xFFFFFFFF) >> 11
    dy = ((tabr >> 5) & 63) - 32
    s = tabr & 31
    assert sorted(e.tolist()) == list(range(n))
    assert (dy == offs[e, 1]).all() and (s == (offs[e, 0] & 31)).all()
    side = 2 * R + 2
    runs = rowsr.reshape(2 * R + 1, 2, side)
    for dz in range(-R, R + 1):
        for sign in (0, 1):  # 0: dx < 0, 1: dx >= 0
            r = runs[dz + R, sign]
            assert (np.diff(r) >= 0).all()
            for y in range(-R, R + 1):
                got = offs[e[r[y + R]:r[y + R + 1]]]
                want = shell[(shell[:, 2] == dz) & (shell[:, 1] == y) & ((shell[:, 0] >= 0) == (sign == 1))]
                assert len(got) == len(want), (dz, sign, y)
                assert (got[:, 2] == dz).all() and (got[:, 1] == y).all()
                assert (np.diff(got[:, 0]) > 0).all()
    # the runs tile the table in order: plane by plane, the dx < 0 run first
    assert runs[0, 0, 0] == 0 and runs[-1, 1, -1] == n
    assert (runs[:, 0, -1] == runs[:, 1, 0]).all() and (runs[1:, 0, 0] == runs[:-1, 1, -1]).all()


def test_row_lane_table_refused_beyond_reach_31(ik):
    with pytest.raises(Exception):
        ik.ik_row_table(40)


@pytest.mark.parametrize("L", [1, 2, 5, 9, 14, 20, 24, 31])
def test_row_mask_table_is_each_offsets_supercover(ik, L):
    """The row-lane edge masks' table (ik_row_mask_table): the voxels listed
    for each offset (in ik_row_table's device order) encode, row delta at
    the halo pitch 32 + 2R and dx, exactly that offset's supercover as
    ik_supercover_offsets builds it."""
    R, offs, _, _ = ik.ik_row_table(L)
    start, tab = ik.ik_row_mask_table(L)
    assert start[0] == 0 and start[-1] == len(tab) and (np.diff(start) >= 0).all()
    RY = 32 + 2 * R
    for e, d in enumerate(offs):
        sc = ik.ik_supercover_offsets(d)
        want = ((sc[:, 2] * RY + sc[:, 1]) << 6) | (sc[:, 0] + 32)
        got = tab[start[e]:start[e + 1]]
        assert sorted(got.tolist()) == sorted(want.tolist()), (L, tuple(d))
        assert (((got & 63) - 32) * np.sign(d[0]) >= 0).all()  # dx of one sign (or 0)
