"""Host logic of the tiled maps, on the CPU: the tile builder's tables.

The tile builder (csrc/layout.cu) cuts the tets, in internal order, into
tiles and packs per tile the corner slots, the reduction entries grouped into
units of at most kUnitEntries, the unit descriptors (slot, run length, run
head) and the slot vertex ids.  The GPU kernels trust these tables, so they
are checked here without a GPU, through a small host driver built from the
same source: tiles partition the tets within the limits, slots name the
corners' vertices, every (tet, corner) entry is summed exactly once by a unit
of its own vertex, runs and heads follow the warp boundaries, and reducing
integer per-corner values through the tables reproduces the per-vertex sums
exactly.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("tiles") / "tile_prefix_dump"
    src = os.path.join(ROOT, "tests", "host", "tile_prefix_dump.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                    "-O1", src, "-o", str(out)], check=True, capture_output=True)
    return str(out)


def _tiles(driver, tmp_path, keys, nv, cap):
    kin, kout = tmp_path / "keys.bin", tmp_path / "prefix.bin"
    with open(kin, "wb") as fh:
        np.array([nv, keys.shape[0], cap], np.int32).tofile(fh)
        np.ascontiguousarray(keys, np.int32).tofile(fh)
    subprocess.run([driver, str(kin), str(kout)], check=True)
    raw = np.fromfile(kout, np.uint8)
    info = raw[:36].view(np.int32)
    ntiles, TT, TS, UE, o_slots, o_ent, o_units, o_vtx, P = (int(x) for x in info)
    blobs = raw[36:].reshape(ntiles, P)
    return dict(TT=TT, TS=TS, UE=UE, o_slots=o_slots, o_ent=o_ent, o_units=o_units, o_vtx=o_vtx, blobs=blobs)


def _check(tb, keys, nv, cap, rng):
    TT, TS, UE = tb["TT"], tb["TS"], tb["UE"]
    nt = keys.shape[0]
    vals = rng.integers(-1000, 1000, size=(nt, 4), dtype=np.int64)       # one value per (tet, corner)
    want = np.zeros(nv, np.int64)
    np.add.at(want, keys.ravel(), vals.ravel())
    got = np.zeros(nv, np.int64)
    seen = np.zeros((nt, 4), np.int32)
    first = 0
    for b in tb["blobs"]:
        ntets, nslots, row0, nunits = (int(x) for x in b[:16].view(np.int32))
        assert row0 == first and 1 <= ntets <= cap
        assert 1 <= nslots <= TS and 1 <= nunits <= TT
        slots = b[tb["o_slots"]:tb["o_slots"] + 4 * TT].reshape(TT, 4).astype(np.int64)
        ent = b[tb["o_ent"]:tb["o_ent"] + 2 * UE * TT].view(np.uint16).reshape(TT, UE)
        units = b[tb["o_units"]:tb["o_units"] + 4 * TT].view(np.uint32)
        vtx = b[tb["o_vtx"]:tb["o_vtx"] + 4 * TS].view(np.int32)
        # slots name the corners' vertices; the slot vertices are distinct
        assert (slots[:ntets] < nslots).all()
        assert np.array_equal(vtx[slots[:ntets]], keys[first:first + ntets])
        assert len(set(vtx[:nslots].tolist())) == nslots
        # unit descriptors: present below nunits only, slot in range
        has = (units & 1).astype(bool)
        assert has[:nunits].all() and not units[nunits:].any()
        uslot = (units >> 14) & 0xFF
        rem = (units >> 22) & 0xF
        head = ((units >> 26) & 1).astype(bool)
        assert (uslot[:nunits] < nslots).all()
        sums = np.zeros(TT, np.int64)
        for i in range(nunits):
            for code in ent[i]:
                if code == 0xFFFF:
                    continue
                a, t = divmod(int(code), 3 * (TT + 1))
                assert a < 4 and t < ntets
                assert slots[t, a] == uslot[i]                 # an entry of the unit's own vertex
                seen[first + t, a] += 1
                sums[i] += vals[first + t, a]
        for i in range(nunits):
            # runs: same slot, same warp; heads start a run
            r = int(rem[i])
            assert i + r < nunits and (i + r) // 32 == i // 32
            assert (uslot[i:i + r + 1] == uslot[i]).all()
            starts = i == 0 or uslot[i - 1] != uslot[i] or i % 32 == 0
            assert head[i] == starts
            if not starts:
                assert rem[i - 1] == r + 1
            if head[i]:
                end = i + r + 1
                assert end == nunits or end % 32 == 0 or uslot[end] != uslot[i]
                got[vtx[uslot[i]]] += sums[i:end].sum()
        first += ntets
    assert first == nt
    assert (seen == 1).all()                                   # every entry summed exactly once
    assert np.array_equal(got, want)                           # the tables reduce exactly


@pytest.mark.parametrize("n,order,cap", [(3, "grid", 128), (5, "grid", 128), (5, "grid", 61), (4, "grid", 1),
                                         (6, "shuffled", 128), (3, "shuffled", 37)])
def test_tile_tables_reduce_every_corner_once(driver, tmp_path, n, order, cap):
    m = meshgen.cube_grid(n, jitter=0.01, seed=n)
    keys = np.asarray(m.tets, np.int32)
    rng = np.random.default_rng(100 + n)
    if order == "shuffled":          # no locality: slot and unit limits cut the tiles
        keys = keys[rng.permutation(keys.shape[0])]
    tb = _tiles(driver, tmp_path, keys, m.n_verts, cap)
    _check(tb, keys, m.n_verts, cap, rng)


def test_runs_across_warps_and_the_unit_limit(driver, tmp_path):
    """Tets (0, 1, 2, k) around a shared triangle: the three shared vertices
    get one unit per 8 of their entries, tiles close on the limit of
    kTileTets units, and the third vertex's run crosses the boundary between
    the first two warps, so a second head must start it there."""
    rng = np.random.default_rng(7)
    nfan = 700
    keys = np.stack([np.zeros(nfan), np.ones(nfan), np.full(nfan, 2), 3 + np.arange(nfan)], axis=1).astype(np.int32)
    nv = 3 + nfan
    tb = _tiles(driver, tmp_path, keys, nv, 128)
    b = tb["blobs"][0]
    nunits = int(b[:16].view(np.int32)[3])
    uslot = (b[tb["o_units"]:tb["o_units"] + 4 * tb["TT"]].view(np.uint32) >> 14) & 0xFF
    assert nunits == tb["TT"] and uslot[31] == uslot[32]      # the case this test is for
    _check(tb, keys, nv, 128, rng)
