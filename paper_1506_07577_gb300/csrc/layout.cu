// Internal layout of a finalized tets relation (host-side construction).
//
// Keys are opaque (Section 5.1, and its footnote: the runtime is free to
// reorder relations), so the library stores tets in its own order:
//   1. Morton order of the tet centroids over the rest shape, which keeps
//      tets that share vertices next to each other;
//   2. tiles of up to kTileTets consecutive tets touching at most kTileSlots
//      distinct vertices, with a tile-local u8 slot per tet corner (the tiled
//      map gathers and pre-reduces through shared memory);
//   3. the inverse of the key-field, vertex -> (tet, corner) entries in CSR
//      form: Section 6.1 groups a relation by a key-field by sorting it and
//      adding a [begin, end) index to the target, which is exactly this.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <numeric>
#include <vector>

#include "ebb_internal.h"

namespace ebb {

namespace {

// Spread the low 21 bits of x to every third bit.
uint64_t spread3(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src, cudaStream_t st) {
  if (src.empty()) {
    *dst = nullptr;
    return cudaSuccess;
  }
  cudaError_t e = cudaMalloc(dst, sizeof(T) * src.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st);
}

}  // namespace

void free_layout(ebb_rel_s* tets) {
  cudaFree(tets->tiles.tet_off);
  cudaFree(tets->tiles.vtx_off);
  cudaFree(tets->tiles.vtx);
  cudaFree(tets->tiles.slots);
  tets->tiles = Tiles();
  cudaFree(tets->vindex.off);
  cudaFree(tets->vindex.ent);
  tets->vindex = VertexIndex();
  cudaFree(tets->tet_perm);
  tets->tet_perm = nullptr;
}

ebb_status_t build_layout(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<int4>& keys,
                          const std::vector<double>& X, std::vector<int>& perm, std::vector<int4>& sorted) {
  const int nt = (int)keys.size();
  const int nv = (int)(X.size() / 3);
  cudaStream_t st = ctx->stream;

  // 1. Morton order of centroids.
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  for (int c = 0; c < 3; ++c) {
    if (nv > 0) {
      auto mm = std::minmax_element(X.begin() + (size_t)c * nv, X.begin() + (size_t)(c + 1) * nv);
      lo[c] = *mm.first;
      hi[c] = *mm.second;
    }
    if (!(hi[c] > lo[c])) hi[c] = lo[c] + 1.0;
  }
  std::vector<std::pair<uint64_t, int>> code(nt);
  const double q = (double)((1u << 21) - 1);
  for (int t = 0; t < nt; ++t) {
    const int k[4] = {keys[t].x, keys[t].y, keys[t].z, keys[t].w};
    uint64_t m = 0;
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int a = 0; a < 4; ++a) s += X[(size_t)c * nv + k[a]];
      double r = (0.25 * s - lo[c]) / (hi[c] - lo[c]);
      r = r < 0 ? 0 : (r > 1 ? 1 : r);
      m |= spread3((uint64_t)(r * q)) << c;
    }
    code[t] = {m, t};
  }
  std::sort(code.begin(), code.end());
  perm.resize(nt);
  sorted.resize(nt);
  for (int i = 0; i < nt; ++i) {
    perm[i] = code[i].second;
    sorted[i] = keys[perm[i]];
  }

  // 2. Tiles.
  std::vector<int> tet_off{0}, vtx_off{0}, vtx;
  std::vector<uchar4> slots(nt);
  std::vector<int> stamp(nv, -1), slot_of(nv, 0);
  int tile = 0, tile_tets = 0, tile_vtx = 0;
  for (int i = 0; i < nt; ++i) {
    const int k[4] = {sorted[i].x, sorted[i].y, sorted[i].z, sorted[i].w};
    int fresh = 0;
    for (int a = 0; a < 4; ++a) fresh += stamp[k[a]] != tile;
    if (tile_tets == kTileTets || tile_vtx + fresh > kTileSlots) {
      tet_off.push_back(i);
      vtx_off.push_back((int)vtx.size());
      ++tile;
      tile_tets = 0;
      tile_vtx = 0;
    }
    unsigned char s[4];
    for (int a = 0; a < 4; ++a) {
      const int v = k[a];
      if (stamp[v] != tile) {
        stamp[v] = tile;
        slot_of[v] = tile_vtx++;
        vtx.push_back(v);
      }
      s[a] = (unsigned char)slot_of[v];
    }
    slots[i] = make_uchar4(s[0], s[1], s[2], s[3]);
    ++tile_tets;
  }
  if (tile_tets > 0) {
    tet_off.push_back(nt);
    vtx_off.push_back((int)vtx.size());
  }
  const int ntiles = (int)tet_off.size() - 1;

  // 3. Vertex -> (tet, corner) index in internal order.
  std::vector<int> voff(nv + 1, 0), vent((size_t)4 * nt);
  for (int i = 0; i < nt; ++i) {
    voff[sorted[i].x + 1]++;
    voff[sorted[i].y + 1]++;
    voff[sorted[i].z + 1]++;
    voff[sorted[i].w + 1]++;
  }
  for (int v = 0; v < nv; ++v) voff[v + 1] += voff[v];
  {
    std::vector<int> fill(voff.begin(), voff.end() - 1);
    for (int i = 0; i < nt; ++i) {
      const int k[4] = {sorted[i].x, sorted[i].y, sorted[i].z, sorted[i].w};
      for (int a = 0; a < 4; ++a) vent[fill[k[a]]++] = 4 * i + a;
    }
  }

  cudaError_t e = upload(&tets->tiles.tet_off, tet_off, st);
  if (e == cudaSuccess) e = upload(&tets->tiles.vtx_off, vtx_off, st);
  if (e == cudaSuccess) e = upload(&tets->tiles.vtx, vtx, st);
  if (e == cudaSuccess) e = upload(&tets->tiles.slots, slots, st);
  if (e == cudaSuccess) e = upload(&tets->vindex.off, voff, st);
  if (e == cudaSuccess) e = upload(&tets->vindex.ent, vent, st);
  if (e == cudaSuccess) e = upload(&tets->tet_perm, perm, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_layout(tets);
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, std::string("building the tet layout: ") + cudaGetErrorString(e));
  }
  tets->tiles.ntiles = ntiles;
  tets->tiles.total_vtx = (int)vtx.size();
  return EBB_OK;
}

}  // namespace ebb
