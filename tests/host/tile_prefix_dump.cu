// CPU driver for the tile builder's host-logic test: reads a key-field in
// internal tet order, cuts it into tiles and writes every tile's blob prefix
// (header, corner slots, reduction entries and units, slot vertex ids), so
// the test can check the tables without a GPU.  No CUDA call is made.
//
//   input : int32 nv, nt, cap, then nt x 4 int32 keys
//   output: int32 ntiles, kTileTets, kTileSlots, kUnitEntries, kBlobSlots,
//           kBlobEnt, kBlobUnits, kBlobVtx, kBlobPrefix, then the prefixes
#include <cstdio>
#include <string>
#include <vector>

#include "../../paper_1506_07577_gb300/csrc/layout.cu"

// Error reporting of the library's other translation units; the tile builder
// never calls them.
namespace ebb {
ebb_status_t set_error(ebb_ctx_s*, int code, const std::string&) { return (ebb_status_t)code; }
ebb_status_t cuda_check(ebb_ctx_s*, cudaError_t e, const char*) { return e == cudaSuccess ? EBB_OK : EBB_ERR_CUDA; }
}  // namespace ebb

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s keys.bin prefix.bin\n", argv[0]);
    return 2;
  }
  FILE* in = std::fopen(argv[1], "rb");
  if (!in) return 3;
  int hdr[3];
  if (std::fread(hdr, sizeof(int), 3, in) != 3) return 4;
  const int nv = hdr[0], nt = hdr[1], cap = hdr[2];
  std::vector<int4> keys(nt);
  if (nt > 0 && std::fread(keys.data(), sizeof(int4), nt, in) != (size_t)nt) return 5;
  std::fclose(in);
  std::vector<unsigned char> prefix;
  const int ntiles = ebb::tile_prefix(keys, nv, cap, prefix);
  FILE* out = std::fopen(argv[2], "wb");
  if (!out) return 6;
  const int info[9] = {ntiles,          ebb::kTileTets, ebb::kTileSlots, ebb::kUnitEntries, ebb::kBlobSlots,
                       ebb::kBlobEnt, ebb::kBlobUnits, ebb::kBlobVtx,   ebb::kBlobPrefix};
  std::fwrite(info, sizeof(int), 9, out);
  if (!prefix.empty()) std::fwrite(prefix.data(), 1, prefix.size(), out);
  std::fclose(out);
  return 0;
}
