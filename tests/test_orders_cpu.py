"""Host logic of finalize, on the CPU: the library's internal orders.

Keys are opaque and the runtime may reorder relations (Section 5.1 and its
footnote), so finalize orders the tets by the Morton code of their centroids
over the rest shape (grouped first by a per-vertex batch id when one is
bound), and EBB_FINALIZE_RENUMBER_VERTS numbers the vertices by the chunks
of tiles that the host-buffer map copies: the vertices of one chunk only,
chunk by chunk, then those several chunks share, then unused ones, each
group in order of first use.  The orders are built by the library's set-up
code (csrc/layout.cu: a radix sort, threads over ranges), run here through a
small host driver; this test recomputes them from those definitions with
numpy sorts and compares them exactly, on meshes with many equal codes.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path_factory, name):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp(name) / name
    src = os.path.join(ROOT, "tests", "host", name + ".cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                    "-O1", src, "-o", str(out)], check=True, capture_output=True)
    return str(out)


@pytest.fixture(scope="module")
def drivers(tmp_path_factory):
    return _build(tmp_path_factory, "orders_dump"), _build(tmp_path_factory, "tile_prefix_dump")


def _run_orders(driver, tmp_path, keys, X, cap=128, nchunks=8, batch=None):
    nt, nv = keys.shape[0], X.shape[0]
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as fh:
        np.array([nv, nt, cap, nchunks, batch is not None], np.int32).tofile(fh)
        np.ascontiguousarray(keys, np.int32).tofile(fh)
        np.ascontiguousarray(X.T, np.float64).tofile(fh)
        if batch is not None:
            np.ascontiguousarray(batch, np.int32).tofile(fh)
    subprocess.run([driver, str(fin), str(fout)], check=True)
    raw = np.fromfile(fout, np.int32)
    out = {"perm": raw[:nt]}
    if batch is None:
        out["own"] = int(raw[nt])
        out["vp"] = raw[nt + 1:nt + 1 + nv]
        out["tperm"] = raw[nt + 1 + nv:]
    return out


def _tile_sizes(driver, tmp_path, sorted_keys, nv, cap):
    kin, kout = tmp_path / "keys.bin", tmp_path / "prefix.bin"
    with open(kin, "wb") as fh:
        np.array([nv, sorted_keys.shape[0], cap], np.int32).tofile(fh)
        np.ascontiguousarray(sorted_keys, np.int32).tofile(fh)
    subprocess.run([driver, str(kin), str(kout)], check=True)
    raw = np.fromfile(kout, np.uint8)
    ntiles, P = int(raw[:4].view(np.int32)[0]), int(raw[32:36].view(np.int32)[0])
    blobs = raw[36:].reshape(ntiles, P)
    return np.array([int(b[:4].view(np.int32)[0]) for b in blobs])


def _spread3(x):
    """The low 21 bits of x moved to every third bit (bit b to bit 3b)."""
    out = np.zeros_like(x)
    for b in range(21):
        out |= ((x >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def _morton_codes(keys, X):
    lo, hi = X.min(axis=0), X.max(axis=0)
    hi = np.where(hi > lo, hi, lo + 1.0)
    q = float((1 << 21) - 1)
    code = np.zeros(keys.shape[0], np.uint64)
    for c in range(3):
        s = np.zeros(keys.shape[0])
        for a in range(4):                       # summed corner by corner, as the definition reads
            s = s + X[keys[:, a], c]
        r = np.clip((0.25 * s - lo[c]) / (hi[c] - lo[c]), 0.0, 1.0)
        code |= _spread3((r * q).astype(np.uint64)) << np.uint64(c)
    return code


def _want_perm(keys, X, batch=None):
    code = _morton_codes(keys, X)
    grp = np.zeros(keys.shape[0], np.int64) if batch is None else batch[keys[:, 0]].astype(np.int64)
    return np.lexsort((np.arange(keys.shape[0]), code, grp))


# The host-buffer map's chunks: 6 of 1, 3, 4, 4, 3 and 1 sixteenths of the
# tiles; any other count cuts evenly.
CHUNK_ENDS = [0, 1, 4, 8, 12, 15, 16]


def _chunk_first_tile(c, ntiles, K):
    if K == len(CHUNK_ENDS) - 1:
        return CHUNK_ENDS[c] * ntiles // CHUNK_ENDS[-1]
    return c * ntiles // K


def _want_vertex_order(sorted_keys, nv, tile_sizes, nchunks):
    nt = sorted_keys.shape[0]
    ntiles = tile_sizes.size
    K = max(1, min(nchunks, ntiles))
    tet_off = np.concatenate([[0], np.cumsum(tile_sizes)])
    chunk_of_tet = np.zeros(nt, np.int64)
    for c in range(K):
        chunk_of_tet[tet_off[_chunk_first_tile(c, ntiles, K)]:tet_off[_chunk_first_tile(c + 1, ntiles, K)]] = c
    fc = np.full(nv, -1)
    lc = np.full(nv, -1)
    first = np.full(nv, nt)
    for t in range(nt):
        for v in sorted_keys[t]:
            if fc[v] < 0:
                fc[v], first[v] = chunk_of_tet[t], t
            lc[v] = chunk_of_tet[t]
    grp = np.where(fc < 0, K + 1, np.where(fc == lc, fc, K))
    vp = np.lexsort((np.arange(nv), first, grp))
    return vp, int((grp < K).sum())


def _tie_heavy(seed, nv=300, nt=900):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 4, size=(nv, 3)).astype(np.float64) * 0.5     # few distinct centroids
    keys = np.array([rng.choice(nv, 4, replace=False) for _ in range(nt)], np.int32)
    return keys, X


CASES = {
    "grid6_shuffled": lambda: (lambda m: (m.tets, m.X))(meshgen.cube_grid(6, jitter=0.01, seed=3, permute=True)),
    "grid5_unjittered": lambda: (lambda m: (m.tets, m.X))(meshgen.cube_grid(5, jitter=0.0, seed=0, permute=True)),
    "tie_heavy": lambda: _tie_heavy(7),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("cap,nchunks", [(128, 6), (37, 6), (37, 3)])
def test_orders_follow_their_definitions(drivers, tmp_path, case, cap, nchunks):
    orders, tiles = drivers
    keys, X = CASES[case]()
    keys = np.ascontiguousarray(keys, np.int32)
    nv = X.shape[0]
    got = _run_orders(orders, tmp_path, keys, X, cap, nchunks)
    want = _want_perm(keys, X)
    assert np.array_equal(got["perm"], want)
    # the vertex order's tet order is the same Morton order
    assert np.array_equal(got["tperm"], want)
    sorted_keys = keys[want]
    vp, own = _want_vertex_order(sorted_keys, nv, _tile_sizes(tiles, tmp_path, sorted_keys, nv, cap), nchunks)
    assert np.array_equal(np.sort(got["vp"]), np.arange(nv))
    assert np.array_equal(got["vp"], vp)
    assert got["own"] == own


def test_batch_ids_group_the_tets_first(drivers, tmp_path):
    orders, _ = drivers
    rng = np.random.default_rng(11)
    keys, X = _tie_heavy(5, nv=200, nt=600)
    batch = rng.integers(0, 5, size=X.shape[0]).astype(np.int32)
    got = _run_orders(orders, tmp_path, keys, X, batch=batch)
    assert np.array_equal(got["perm"], _want_perm(keys, X, batch))
    g = batch[keys[got["perm"], 0]]
    assert (np.diff(g) >= 0).all()
