// CPU driver for the host-logic test of the internal orders: the Morton
// order of the tets (optionally grouped by a per-vertex batch id) and the
// chunk-grouped vertex order of EBB_FINALIZE_RENUMBER_VERTS, computed by the
// library's own set-up code (csrc/layout.cu) on the host.  No CUDA call is
// made.
//
//   input : int32 nv, nt, cap, nchunks, has_batch, then nt x 4 int32 keys,
//           3 x nv float64 rest positions (planes), nv int32 batch ids
//           (if has_batch)
//   output: int32 perm[nt] (tet_morton_order), then, without batch ids,
//           int32 own, vp[nv], tperm[nt] (chunked_vertex_order)
#include <cstdio>
#include <string>
#include <vector>

#include "../../paper_1506_07577_gb300/csrc/layout.cu"

// Error reporting of the library's other translation units; these orders
// never call them.
namespace ebb {
ebb_status_t set_error(ebb_ctx_s*, int code, const std::string&) { return (ebb_status_t)code; }
ebb_status_t cuda_check(ebb_ctx_s*, cudaError_t e, const char*) { return e == cudaSuccess ? EBB_OK : EBB_ERR_CUDA; }
}  // namespace ebb

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]);
    return 2;
  }
  FILE* in = std::fopen(argv[1], "rb");
  if (!in) return 3;
  int hdr[5];
  if (std::fread(hdr, sizeof(int), 5, in) != 5) return 4;
  const int nv = hdr[0], nt = hdr[1], cap = hdr[2], nchunks = hdr[3], has_batch = hdr[4];
  std::vector<int4> keys(nt);
  std::vector<double> X((size_t)3 * nv);
  std::vector<int> batch(has_batch ? nv : 0);
  if (nt > 0 && std::fread(keys.data(), sizeof(int4), nt, in) != (size_t)nt) return 5;
  if (nv > 0 && std::fread(X.data(), sizeof(double), X.size(), in) != X.size()) return 6;
  if (has_batch && nv > 0 && std::fread(batch.data(), sizeof(int), nv, in) != (size_t)nv) return 7;
  std::fclose(in);
  std::vector<int> perm;
  ebb::tet_morton_order(keys, X, has_batch ? &batch : nullptr, perm);
  FILE* out = std::fopen(argv[2], "wb");
  if (!out) return 8;
  std::fwrite(perm.data(), sizeof(int), perm.size(), out);
  if (!has_batch) {
    std::vector<int> vp, tperm;
    int own = -1;
    ebb::chunked_vertex_order(keys, X, cap, nchunks, vp, &own, &tperm);
    std::fwrite(&own, sizeof(int), 1, out);
    std::fwrite(vp.data(), sizeof(int), vp.size(), out);
    std::fwrite(tperm.data(), sizeof(int), tperm.size(), out);
  }
  std::fclose(out);
  return 0;
}
