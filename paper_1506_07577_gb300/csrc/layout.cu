// Internal layout of a finalized tets relation.
//
// Keys are opaque (Section 5.1, and its footnote: the runtime is free to
// reorder relations), so the library stores tets in its own order:
//   1. Morton order of the tet centroids over the rest shape, which keeps
//      tets that share vertices next to each other (grouped first by the
//      optional per-vertex batch id, so independent meshes stay apart);
//   2. tiles of up to kTileTets consecutive tets touching at most kTileSlots
//      distinct vertices; each tile's data is packed into one contiguous blob
//      (see ebb_internal.h) that the tiled map fetches with one bulk copy;
//   3. the inverse of the key-field, vertex -> (tet, corner) entries in CSR
//      form: Section 6.1 groups a relation by a key-field by sorting it and
//      adding a [begin, end) index to the target, which is exactly this.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <tuple>
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

// Order the entries of the reduction units of 16 consecutive threads (one
// half-warp) over the kUnitEntries steps so that, at each step, the threads
// read output rows in distinct shared-memory bank pairs.  The bank pair of
// the row coded 3a*(kTileTets+1) + t is code mod 16 (kTileTets+1 = 1 mod 16).
// This is an edge colouring of the bipartite multigraph threads x bank pairs
// with one colour per step: with every degree at most kUnitEntries it exists
// (Koenig's edge-colouring theorem) and the alternating-path method finds it.
// A bank pair with more than kUnitEntries entries is first split into copies
// of at most kUnitEntries each (entries of different copies may then share a
// step: the unavoidable conflicts).  ent[l * kUnitEntries + q] receives the
// entry thread l reads at step q, or kEntryNone.
void schedule_half_warp(std::vector<std::vector<unsigned short>>& lanes, unsigned short* ent) {
  constexpr int C = kUnitEntries;
  const int nl = (int)lanes.size();
  struct Edge {
    int x, y, colour;
    unsigned short code;
  };
  std::vector<Edge> edges;
  int copies[16] = {0}, fill[16] = {0}, first_copy[16];
  for (int l = 0; l < nl; ++l)
    for (unsigned short code : lanes[l]) copies[code & 15]++;
  int nright = 0;
  for (int k = 0; k < 16; ++k) {
    first_copy[k] = nright;
    nright += (copies[k] + C - 1) / C;
  }
  for (int l = 0; l < nl; ++l)
    for (unsigned short code : lanes[l]) {
      const int k = code & 15;
      edges.push_back({l, nl + first_copy[k] + fill[k]++ / C, -1, code});
    }
  const int nvert = nl + nright;
  std::vector<int> at((size_t)nvert * C, -1);  // at[v*C + colour] = edge
  auto free_colour = [&](int v) {
    for (int c = 0; c < C; ++c)
      if (at[(size_t)v * C + c] < 0) return c;
    return -1;
  };
  for (int e = 0; e < (int)edges.size(); ++e) {
    const int x = edges[e].x, y = edges[e].y;
    const int a = free_colour(x), b = free_colour(y);
    if (at[(size_t)y * C + a] >= 0) {
      // Swap colours a and b along the path from y that alternates a, b.
      std::vector<int> path;
      int v = y, c = a;
      while (at[(size_t)v * C + c] >= 0) {
        const int f = at[(size_t)v * C + c];
        path.push_back(f);
        v = edges[f].x == v ? edges[f].y : edges[f].x;
        c = c == a ? b : a;
      }
      for (int f : path) {
        at[(size_t)edges[f].x * C + edges[f].colour] = -1;
        at[(size_t)edges[f].y * C + edges[f].colour] = -1;
      }
      for (int f : path) {
        edges[f].colour = edges[f].colour == a ? b : a;
        at[(size_t)edges[f].x * C + edges[f].colour] = f;
        at[(size_t)edges[f].y * C + edges[f].colour] = f;
      }
    }
    edges[e].colour = a;
    at[(size_t)x * C + a] = e;
    at[(size_t)y * C + a] = e;
  }
  for (int i = 0; i < nl * C; ++i) ent[i] = kEntryNone;
  for (const Edge& e : edges) ent[e.x * C + e.colour] = e.code;
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

// Blob layout for one precision.  The stride between blobs (and a ring
// stage) holds the larger of the two record layouts, so that switching
// between them needs no reallocation; a kernel copies only what the chosen
// layout uses (planes without per-tet material stop after the V plane).
BlobLayout make_layout(size_t elem, bool material, bool planes) {
  BlobLayout L;
  L.rec = kBlobPrefix;
  L.material = material;
  L.planes = planes;
  const int rl = elem == 4 ? rec_len<float>() : rec_len<double>();
  const int rows_end = L.rec + (int)(kTileTets * rl * elem);
  const int planes_end = L.rec + (int)(kTileTets * (material ? 12 : 10) * elem);
  const int end = planes ? planes_end : rows_end;
  L.copy = (end + 15) / 16 * 16;
  L.bytes = (std::max(rows_end, L.rec + (int)(kTileTets * 12 * elem)) + 127) / 128 * 128;
  return L;
}

// One CTA per tile: copy the integer prefix (unless `prefix` is null: the
// blob holds it already), then gather the tile's per-tet element-precision
// values from the planar streams into the records (zero past the tile end).
template <typename T>
__global__ void pack_blob_kernel(int nt, const unsigned char* __restrict__ prefix, TetStreams<T> s, BlobLayout L,
                                 unsigned char* blob) {
  const int tile = blockIdx.x;
  unsigned char* b = blob + (size_t)tile * L.bytes;
  if (prefix != nullptr) {
    const int4* src = reinterpret_cast<const int4*>(prefix + (size_t)tile * kBlobPrefix);
    int4* dst = reinterpret_cast<int4*>(b);
    for (int i = threadIdx.x; i < kBlobPrefix / 16; i += blockDim.x) dst[i] = src[i];
  }
  const int4 hdr = prefix != nullptr ? reinterpret_cast<const int4*>(prefix + (size_t)tile * kBlobPrefix)[0]
                                     : reinterpret_cast<const int4*>(b)[0];
  const int ntets = hdr.x, tb = hdr.z;
  T* R = reinterpret_cast<T*>(b + L.rec);
  for (int i = threadIdx.x; i < kTileTets; i += blockDim.x) {
    const bool in = i < ntets;
    const int t = tb + i;
    T v[12];
    for (int k = 0; k < 9; ++k) v[k] = in ? s.B[(size_t)k * nt + t] : T(0);
    v[9] = in ? s.V[t] : T(0);
    v[10] = (in && L.material) ? s.mu[t] : T(0);
    v[11] = (in && L.material) ? s.lam[t] : T(0);
    if (L.planes) {
      for (int k = 0; k < 12; ++k) R[(size_t)k * kTileTets + i] = v[k];
    } else {
      constexpr int RL = rec_len<T>();
      T* r = R + (size_t)RL * i;
      for (int k = 0; k < 12; ++k) r[k] = v[k];
      for (int k = 12; k < RL; ++k) r[k] = T(0);
    }
  }
}

}  // namespace

// Tiles: greedy cut of the internal (Morton) tet order.  A tile closes before
// it would exceed `cap` tets, kTileSlots distinct vertices, kTileTets
// reduction units (ceil(entries / kUnitEntries) summed over its vertices) or
// kUnitMaxRun units for one vertex.  The cut depends on which corners share
// a vertex, not on the vertex numbers.  Returns the tile boundaries
// (ntiles + 1 entries).
std::vector<int> tile_cut(const std::vector<int4>& sorted, int nv, int cap) {
  const int nt = (int)sorted.size();
  std::vector<int> tet_off{0};
  {
    std::vector<int> stamp(nv, -1), count(nv, 0);
    int tile = 0, tile_tets = 0, tile_vtx = 0, tile_units = 0;
    for (int i = 0; i < nt; ++i) {
      const int k[4] = {sorted[i].x, sorted[i].y, sorted[i].z, sorted[i].w};
      int fresh = 0, more_units = 0;
      bool run_ok = true;
      for (int a = 0; a < 4; ++a) {
        const int c = stamp[k[a]] == tile ? count[k[a]] : 0;
        fresh += c == 0;
        more_units += c % kUnitEntries == 0;
        run_ok = run_ok && (c + 1 + kUnitEntries - 1) / kUnitEntries <= kUnitMaxRun;
      }
      if (tile_tets == cap || tile_vtx + fresh > kTileSlots || tile_units + more_units > kTileTets ||
          !run_ok) {
        tet_off.push_back(i);
        ++tile;
        tile_tets = tile_vtx = tile_units = 0;
      }
      for (int a = 0; a < 4; ++a) {
        if (stamp[k[a]] != tile) {
          stamp[k[a]] = tile;
          count[k[a]] = 0;
          ++tile_vtx;
        }
        if (count[k[a]] % kUnitEntries == 0) ++tile_units;
        ++count[k[a]];
      }
      ++tile_tets;
    }
    if (tile_tets > 0) tet_off.push_back(nt);
  }
  return tet_off;
}

namespace {

// Cut the internal tet order into tiles of at most `cap` tets and build each
// tile's blob prefix; returns the tile count.
// Vertex -> per-tile value (open addressing; a tile holds at most
// kTileSlots vertices), so that building one tile touches only its own few
// kilobytes whatever the vertex numbering.
struct TileVertexMap {
  static constexpr int kBits = 9;
  static constexpr int kSize = 1 << kBits;
  static_assert(kSize >= 2 * kTileSlots, "load factor");
  int key[kSize];
  int val[kSize];
  void clear() { std::fill(key, key + kSize, -1); }
  // The value of vertex v (>= 0), inserted as -1 when absent.
  int& operator[](int v) {
    unsigned h = ((unsigned)v * 2654435761u) >> (32 - kBits);
    while (key[h] != v) {
      if (key[h] < 0) {
        key[h] = v;
        val[h] = -1;
        break;
      }
      h = (h + 1) & (kSize - 1);
    }
    return val[h];
  }
};

int tile_prefix(const std::vector<int4>& sorted, int nv, int cap, std::vector<unsigned char>& prefix) {
  const std::vector<int> tet_off = tile_cut(sorted, nv, cap);
  const int ntiles = (int)tet_off.size() - 1;

  // Blob prefix per tile: slots (numbered by decreasing entry count), the
  // entries grouped by slot, the reduction units and the vertex ids.
  prefix.assign((size_t)ntiles * kBlobPrefix, 0);
  // Tiles are independent: host threads take contiguous ranges of them,
  // each with scratch of its own.
  parallel_ranges(ntiles, 512, [&](int lo, int hi) {
    TileVertexMap slot_of;
    std::vector<int> vtx, rk, label, member_off, members;
    std::vector<long> grp_count;
    std::vector<int> cnt(kTileSlots + 1);
    for (int ti = lo; ti < hi; ++ti) {
      unsigned char* b = prefix.data() + (size_t)ti * kBlobPrefix;
      uchar4* slots = reinterpret_cast<uchar4*>(b + kBlobSlots);
      unsigned short* ent = reinterpret_cast<unsigned short*>(b + kBlobEnt);
      uint32_t* units = reinterpret_cast<uint32_t*>(b + kBlobUnits);
      int* bvtx = reinterpret_cast<int*>(b + kBlobVtx);
      const int tb = tet_off[ti], te = tet_off[ti + 1];
      vtx.clear();
      slot_of.clear();
      for (int t = tb; t < te; ++t) {
        const int k[4] = {sorted[t].x, sorted[t].y, sorted[t].z, sorted[t].w};
        for (int a = 0; a < 4; ++a) {
          int& c = slot_of[k[a]];
          if (c < 0) {
            c = 0;
            vtx.push_back(k[a]);
          }
          c++;
        }
      }
      std::stable_sort(vtx.begin(), vtx.end(), [&](int x, int y) { return slot_of[x] > slot_of[y]; });
      // Rank j = position by decreasing entry count (the reduction units
      // follow this order).
      for (size_t j = 0; j < vtx.size(); ++j) slot_of[vtx[j]] = (int)j;
      const int nvu = (int)vtx.size();
      const int T = te - tb;
      rk.resize((size_t)4 * T);
      for (int t = tb; t < te; ++t) {
        const int k[4] = {sorted[t].x, sorted[t].y, sorted[t].z, sorted[t].w};
        for (int a = 0; a < 4; ++a) rk[(size_t)4 * (t - tb) + a] = slot_of[k[a]];
      }
      // Slot labels: phase 1 reads slot vectors (16 bytes each) for corner a
      // of 8 consecutive tets per shared-memory wavefront, conflict-free when
      // their distinct slots differ mod 8.  Each rank gets the residue class
      // that adds the fewest collisions over the (8 tets, corner) groups it
      // belongs to (greedy, in rank order), with the labels kept compact:
      // class c holds the labels c, c + 8, ... below nvu.
      {
        const int ngroups = ((T + 7) / 8) * 4;
        grp_count.assign((size_t)ngroups * 8, 0);
        member_off.assign(nvu + 1, 0);
        for (int g = 0; g < ngroups; ++g) {
          const int q0 = (g / 4) * 8, a = g % 4;
          for (int t = q0; t < std::min(T, q0 + 8); ++t) {
            const int r = rk[(size_t)4 * t + a];
            bool seen = false;
            for (int t2 = q0; t2 < t; ++t2) seen = seen || rk[(size_t)4 * t2 + a] == r;
            if (!seen) member_off[r + 1]++;
          }
        }
        for (int r = 0; r < nvu; ++r) member_off[r + 1] += member_off[r];
        members.resize(member_off[nvu]);
        std::vector<int> fillm(member_off.begin(), member_off.end() - 1);
        for (int g = 0; g < ngroups; ++g) {
          const int q0 = (g / 4) * 8, a = g % 4;
          for (int t = q0; t < std::min(T, q0 + 8); ++t) {
            const int r = rk[(size_t)4 * t + a];
            bool seen = false;
            for (int t2 = q0; t2 < t; ++t2) seen = seen || rk[(size_t)4 * t2 + a] == r;
            if (!seen) members[fillm[r]++] = g;
          }
        }
        int used[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        label.resize(nvu);
        for (int r = 0; r < nvu; ++r) {
          int best = -1;
          long bestc = 0;
          for (int c = 0; c < 8; ++c) {
            const int cap = nvu > c ? (nvu - c + 7) / 8 : 0;
            if (used[c] >= cap) continue;
            long cost = 0;
            for (int i = member_off[r]; i < member_off[r + 1]; ++i) cost += grp_count[(size_t)members[i] * 8 + c];
            if (best < 0 || cost < bestc) {
              best = c;
              bestc = cost;
            }
          }
          label[r] = best + 8 * used[best]++;
          for (int i = member_off[r]; i < member_off[r + 1]; ++i) grp_count[(size_t)members[i] * 8 + best]++;
        }
      }
      for (int t = 0; t < T; ++t)
        slots[t] = make_uchar4((unsigned char)label[rk[(size_t)4 * t]], (unsigned char)label[rk[(size_t)4 * t + 1]],
                               (unsigned char)label[rk[(size_t)4 * t + 2]],
                               (unsigned char)label[rk[(size_t)4 * t + 3]]);
      std::fill(cnt.begin(), cnt.end(), 0);
      for (size_t i = 0; i < (size_t)4 * T; ++i) cnt[rk[i] + 1]++;
      for (int j = 0; j < nvu; ++j) cnt[j + 1] += cnt[j];
      // Units: thread i sums a run of <= kUnitEntries entries of one vertex
      // (ranks in order).  Consecutive units of a vertex inside one warp form
      // a segment combined by shuffles; its first lane adds the sum into the
      // field.
      std::vector<unsigned short> grouped(cnt[nvu]);
      {
        std::vector<int> fill(cnt.begin(), cnt.begin() + nvu);
        for (int t = 0; t < T; ++t)
          for (int a = 0; a < 4; ++a)
            grouped[fill[rk[(size_t)4 * t + a]]++] = (unsigned short)(3 * a * (kTileTets + 1) + t);
      }
      int nunits = 0;
      std::vector<int> uslot;
      std::vector<std::vector<unsigned short>> unit_ent;
      for (int j = 0; j < nvu; ++j) {
        for (int e = cnt[j]; e < cnt[j + 1]; e += kUnitEntries) {
          const int n = std::min(kUnitEntries, cnt[j + 1] - e);
          unit_ent.emplace_back(grouped.begin() + e, grouped.begin() + e + n);
          units[nunits] = 1u | ((uint32_t)label[j] << 14);
          uslot.push_back(j);
          ++nunits;
        }
      }
      for (int h0 = 0; h0 < nunits; h0 += 16) {
        std::vector<std::vector<unsigned short>> half(unit_ent.begin() + h0,
                                                      unit_ent.begin() + std::min(nunits, h0 + 16));
        schedule_half_warp(half, ent + h0 * kUnitEntries);
      }
      for (int i = 0; i < nunits; ++i) {
        const bool head = i == 0 || uslot[i - 1] != uslot[i] || (i % 32) == 0;
        int last = i;
        while (last + 1 < nunits && uslot[last + 1] == uslot[i] && (last + 1) % 32 != 0) ++last;
        units[i] |= ((uint32_t)(last - i) << 22) | ((uint32_t)head << 26);
      }
      for (int j = 0; j < nvu; ++j) bvtx[label[j]] = vtx[j];
      int* hdr = reinterpret_cast<int*>(b);
      hdr[0] = te - tb;
      hdr[1] = nvu;
      hdr[2] = tb;
      hdr[3] = nunits;
    }
  });

  return ntiles;
}

}  // namespace

// Free the tile blobs and the partial index (not the tile count).
void free_tiles(Tiles& tl) {
  cudaFree(tl.blob32);
  cudaFree(tl.blob64);
  cudaFree(tl.ord_off);
  cudaFree(tl.ord_vtx);
  cudaFree(tl.unit_row);
  cudaFree(tl.partial[0]);
  cudaFree(tl.partial[1]);
  const int n = tl.ntiles;
  tl = Tiles();
  tl.ntiles = n;
}

void free_layout(ebb_rel_s* tets) {
  free_tiles(tets->tiles);
  tets->tiles = Tiles();
  cudaFree(tets->vindex.off);
  cudaFree(tets->vindex.ent);
  cudaFree(tets->vindex.order);
  tets->vindex = VertexIndex();
  cudaFree(tets->tet_perm);
  tets->tet_perm = nullptr;
}

void radix_order(const std::vector<uint64_t>& key, int bits, std::vector<int>& order) {
  const int n = (int)key.size();
  if (order.empty()) {
    order.resize(n);
    for (int i = 0; i < n; ++i) order[i] = i;
  }
  constexpr int kDigit = 11, kBuckets = 1 << kDigit;
  // Each pass: per-block digit counts, their exclusive sums in (digit,
  // block) order, then every block scatters its items in item order; the
  // blocks are fixed ranges of the input, so the result does not depend on
  // the thread count.
  const int nblk = std::max(1, std::min(64, n / (1 << 15)));
  auto blk_lo = [&](int b) { return (int)((long long)n * b / nblk); };
  std::vector<uint64_t> k0(n), k1(n);
  std::vector<int> i1(n);
  for (int i = 0; i < n; ++i) k0[i] = key[order[i]];
  std::vector<int> count((size_t)nblk * kBuckets);
  for (int shift = 0; shift < bits; shift += kDigit) {
    parallel_ranges(nblk, 1, [&](int b0, int b1) {
      for (int b = b0; b < b1; ++b) {
        int* c = count.data() + (size_t)b * kBuckets;
        std::fill(c, c + kBuckets, 0);
        for (int i = blk_lo(b); i < blk_lo(b + 1); ++i) c[(k0[i] >> shift) & (kBuckets - 1)]++;
      }
    });
    bool moves = true;
    {
      const unsigned d0 = n ? (unsigned)((k0[0] >> shift) & (kBuckets - 1)) : 0u;
      int same = 0;
      for (int b = 0; b < nblk; ++b) same += count[(size_t)b * kBuckets + d0];
      moves = same != n;  // one digit value: nothing moves
    }
    if (!moves) continue;
    int run = 0;
    for (int d = 0; d < kBuckets; ++d)
      for (int b = 0; b < nblk; ++b) {
        int& c = count[(size_t)b * kBuckets + d];
        const int x = c;
        c = run;
        run += x;
      }
    parallel_ranges(nblk, 1, [&](int b0, int b1) {
      for (int b = b0; b < b1; ++b) {
        int* c = count.data() + (size_t)b * kBuckets;
        for (int i = blk_lo(b); i < blk_lo(b + 1); ++i) {
          const int d = c[(k0[i] >> shift) & (kBuckets - 1)]++;
          k1[d] = k0[i];
          i1[d] = order[i];
        }
      }
    });
    k0.swap(k1);
    order.swap(i1);
  }
}

void tet_morton_order(const std::vector<int4>& keys, const std::vector<double>& X, const std::vector<int>* batch,
                      std::vector<int>& perm) {
  const int nt = (int)keys.size();
  const int nv = (int)(X.size() / 3);
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  for (int c = 0; c < 3; ++c) {
    if (nv > 0) {
      auto mm = std::minmax_element(X.begin() + (size_t)c * nv, X.begin() + (size_t)(c + 1) * nv);
      lo[c] = *mm.first;
      hi[c] = *mm.second;
    }
    if (!(hi[c] > lo[c])) hi[c] = lo[c] + 1.0;
  }
  // Order: (group id, Morton code of the centroid, row).
  std::vector<uint64_t> code(nt);
  const double q = (double)((1u << 21) - 1);
  parallel_ranges(nt, 1 << 16, [&](int t0, int t1) {
    for (int t = t0; t < t1; ++t) {
      const int k[4] = {keys[t].x, keys[t].y, keys[t].z, keys[t].w};
      uint64_t m = 0;
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int a = 0; a < 4; ++a) s += X[(size_t)c * nv + k[a]];
        double r = (0.25 * s - lo[c]) / (hi[c] - lo[c]);
        r = r < 0 ? 0 : (r > 1 ? 1 : r);
        m |= spread3((uint64_t)(r * q)) << c;
      }
      code[t] = m;
    }
  });
  perm.clear();
  radix_order(code, 63, perm);
  if (batch) {
    // group ids are non-negative (checked at finalize)
    for (int t = 0; t < nt; ++t) code[t] = (uint32_t)(*batch)[keys[t].x];
    radix_order(code, 32, perm);
  }
}

void chunked_vertex_order(const std::vector<int4>& keys, const std::vector<double>& X, int cap, int nchunks,
                          std::vector<int>& vp, int* n_own, std::vector<int>* tperm_out) {
  const int nt = (int)keys.size();
  const int nv = (int)(X.size() / 3);
  std::vector<int> tperm;
  tet_morton_order(keys, X, nullptr, tperm);
  std::vector<int4> sorted(nt);
  for (int i = 0; i < nt; ++i) sorted[i] = keys[tperm[i]];
  const std::vector<int> tet_off = tile_cut(sorted, nv, cap);
  const int ntiles = (int)tet_off.size() - 1;
  const int K = std::max(1, std::min(nchunks, ntiles));
  // first and last chunk of every vertex, and its first tet
  std::vector<int> fc(nv, -1), lc(nv, -1), first(nv, nt);
  for (int c = 0; c < K; ++c) {
    const int t0 = tet_off[(size_t)chunk_first_tile(c, ntiles, K)];
    const int t1 = tet_off[(size_t)chunk_first_tile(c + 1, ntiles, K)];
    for (int t = t0; t < t1; ++t) {
      const int k[4] = {sorted[t].x, sorted[t].y, sorted[t].z, sorted[t].w};
      for (int a = 0; a < 4; ++a) {
        if (fc[k[a]] < 0) {
          fc[k[a]] = c;
          first[k[a]] = t;
        }
        lc[k[a]] = c;
      }
    }
  }
  // rows: the vertices of one chunk only, chunk by chunk, then the vertices
  // several chunks share, then unreferenced ones; each group in the order of
  // first use (ties within a tet by vertex number), unreferenced ones by
  // number.  Built by one pass over the tets in order.
  std::vector<std::vector<int>> group(K + 2);
  for (int t = 0; t < nt; ++t) {
    int k[4] = {sorted[t].x, sorted[t].y, sorted[t].z, sorted[t].w};
    std::sort(k, k + 4);
    for (int a = 0; a < 4; ++a)
      if (first[k[a]] == t) group[fc[k[a]] == lc[k[a]] ? fc[k[a]] : K].push_back(k[a]);
  }
  for (int v = 0; v < nv; ++v)
    if (fc[v] < 0) group[K + 1].push_back(v);
  vp.clear();
  vp.reserve(nv);
  for (int g = 0; g < K + 2; ++g) {
    vp.insert(vp.end(), group[g].begin(), group[g].end());
    if (g == K - 1) *n_own = (int)vp.size();
  }
  if (tperm_out) tperm_out->swap(tperm);
}

ebb_status_t build_layout(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<int4>& keys,
                          const std::vector<double>& X, const std::vector<int>* batch, std::vector<int>& perm,
                          std::vector<int4>& sorted, std::vector<unsigned char>& prefix,
                          const std::vector<int>* known_perm) {
  const int nt = (int)keys.size();
  const int nv = (int)(X.size() / 3);
  cudaStream_t st = ctx->stream;

  // 1. Morton order of centroids.
  if (known_perm && (int)known_perm->size() == nt)
    perm = *known_perm;
  else
    tet_morton_order(keys, X, batch, perm);
  sorted.resize(nt);
  for (int i = 0; i < nt; ++i) sorted[i] = keys[perm[i]];

  // 2. Vertex -> (tet, corner) index in internal order.
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

  // Vertices by first entry (= first use by the internal tets), unused ones
  // last in number order.
  std::vector<int> vorder;
  vorder.reserve(nv);
  {
    std::vector<unsigned char> seen(nv, 0);
    for (int i = 0; i < nt; ++i) {
      const int k[4] = {sorted[i].x, sorted[i].y, sorted[i].z, sorted[i].w};
      for (int a = 0; a < 4; ++a)
        if (!seen[k[a]]) {
          seen[k[a]] = 1;
          vorder.push_back(k[a]);
        }
    }
    for (int v = 0; v < nv; ++v)
      if (!seen[v]) vorder.push_back(v);
  }

  const int ntiles = tile_prefix(sorted, nv, tets->tile_cap, prefix);

  cudaError_t e = upload(&tets->vindex.off, voff, st);
  if (e == cudaSuccess) e = upload(&tets->vindex.ent, vent, st);
  if (e == cudaSuccess) e = upload(&tets->vindex.order, vorder, st);
  if (e == cudaSuccess) e = upload(&tets->tet_perm, perm, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_layout(tets);
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, std::string("building the tet layout: ") + cudaGetErrorString(e));
  }
  tets->tiles.ntiles = ntiles;
  return EBB_OK;
}

ebb_status_t rebuild_tiles(ebb_ctx_s* ctx, ebb_rel_s* tets, int cap) {
  if (cap < 1 || cap > kTileTets) return set_error(ctx, EBB_ERR_ARG, "tile size out of range");
  const int nt = (int)tets->size;
  const int nv = (int)tets->verts->size;
  std::vector<int4> sorted(nt);
  cudaError_t e = cudaSuccess;
  if (nt > 0) e = cudaMemcpyAsync(sorted.data(), tets->keys, sizeof(int4) * nt, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "reading internal keys");
  std::vector<unsigned char> prefix;
  const int ntiles = tile_prefix(sorted, nv, cap, prefix);
  free_tiles(tets->tiles);
  tets->tiles = Tiles();
  tets->tiles.ntiles = ntiles;
  tets->tile_cap = cap;
  ++tets->layout_gen;
  return build_tile_blobs(ctx, tets, prefix);
}

ebb_status_t repack_records(ebb_ctx_s* ctx, ebb_rel_s* tets, bool planes) {
  Tiles& tl = tets->tiles;
  tets->rec_planes = planes;
  if (tl.ntiles == 0) return EBB_OK;
  const bool material = tets->s64.mu != nullptr;
  tl.L32 = make_layout(sizeof(float), material, planes);
  tl.L64 = make_layout(sizeof(double), material, planes);
  const int nt = (int)tets->size;
  pack_blob_kernel<float><<<tl.ntiles, 256, 0, ctx->stream>>>(nt, nullptr, tets->s32, tl.L32, tl.blob32);
  pack_blob_kernel<double><<<tl.ntiles, 256, 0, ctx->stream>>>(nt, nullptr, tets->s64, tl.L64, tl.blob64);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "repacking tile records");
  ++tets->layout_gen;
  return EBB_OK;
}

ebb_status_t build_tile_blobs(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<unsigned char>& prefix) {
  Tiles& tl = tets->tiles;
  const int ntiles = tl.ntiles;
  if (ntiles == 0) return EBB_OK;
  cudaStream_t st = ctx->stream;
  {
    // Partial-row index of the ordered tiled variant: vertices in order of
    // first use by the run-head units (tile by tile), each vertex's rows
    // consecutive and in tile order.
    const int nv = (int)tets->verts->size;
    std::vector<int> pos(nv, -1), ord_vtx, count;
    for (int t = 0; t < ntiles; ++t) {
      const unsigned char* b = prefix.data() + (size_t)t * kBlobPrefix;
      const uint32_t* units = reinterpret_cast<const uint32_t*>(b + kBlobUnits);
      const int* bvtx = reinterpret_cast<const int*>(b + kBlobVtx);
      for (int i = 0; i < kTileTets; ++i) {
        if (!((units[i] >> 26) & 1u)) continue;
        const int v = bvtx[(units[i] >> 14) & 0xffu];
        if (pos[v] < 0) {
          pos[v] = (int)ord_vtx.size();
          ord_vtx.push_back(v);
          count.push_back(0);
        }
        ++count[pos[v]];
      }
    }
    std::vector<int> ord_off(ord_vtx.size() + 1, 0);
    for (size_t k = 0; k < ord_vtx.size(); ++k) ord_off[k + 1] = ord_off[k] + count[k];
    std::vector<int> unit_row((size_t)ntiles * kTileTets, -1);
    {
      std::vector<int> fill(ord_off.begin(), ord_off.end() - 1);
      for (int t = 0; t < ntiles; ++t) {
        const unsigned char* b = prefix.data() + (size_t)t * kBlobPrefix;
        const uint32_t* units = reinterpret_cast<const uint32_t*>(b + kBlobUnits);
        const int* bvtx = reinterpret_cast<const int*>(b + kBlobVtx);
        for (int i = 0; i < kTileTets; ++i) {
          if (!((units[i] >> 26) & 1u)) continue;
          const int v = bvtx[(units[i] >> 14) & 0xffu];
          unit_row[(size_t)t * kTileTets + i] = fill[pos[v]]++;
        }
      }
    }
    tl.n_ord = (int)ord_vtx.size();
    cudaError_t e = upload(&tl.ord_off, ord_off, st);
    if (e == cudaSuccess) e = upload(&tl.ord_vtx, ord_vtx, st);
    if (e == cudaSuccess) e = upload(&tl.unit_row, unit_row, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the tile partial index failed");
    }
  }
  const bool material = tets->s64.mu != nullptr;
  tl.L32 = make_layout(sizeof(float), material, tets->rec_planes);
  tl.L64 = make_layout(sizeof(double), material, tets->rec_planes);
  unsigned char* dprefix = nullptr;
  cudaError_t e = upload(&dprefix, prefix, st);
  if (e == cudaSuccess) e = cudaMalloc(&tl.blob32, (size_t)ntiles * tl.L32.bytes);
  if (e == cudaSuccess) e = cudaMalloc(&tl.blob64, (size_t)ntiles * tl.L64.bytes);
  if (e == cudaSuccess) {
    const int nt = (int)tets->size;
    pack_blob_kernel<float><<<ntiles, 256, 0, st>>>(nt, dprefix, tets->s32, tl.L32, tl.blob32);
    pack_blob_kernel<double><<<ntiles, 256, 0, st>>>(nt, dprefix, tets->s64, tl.L64, tl.blob64);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dprefix);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, std::string("packing tile blobs: ") + cudaGetErrorString(e));
  }
  return EBB_OK;
}

}  // namespace ebb
