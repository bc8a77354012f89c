// P16 link-storage instantiations of the half operator with FP32 Krylov
// vectors (the default solver and the operator calls of the C ABI); the
// P16-vector ones (STAG_HALF_VECTORS, STAG_ROUND_OUTPUT) are in
// dslash_p16h.cu, compiled in parallel.
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p16h(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                               cudaStream_t st, const DsArgs &a, const void **kptr);

cudaError_t launch_dslash_p16(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(P16, 0, P32, P32, 1)
  STAG_DS_EPIS(P16, 0, P32, P32, 4)
  STAG_DS_EPIS(P16, 0, P32, P32, 8)
  STAG_DS_EPIS(P16, 1, P32, P32, 1)
  STAG_DS_EPIS(P16, 1, P32, P32, 4)
  STAG_DS_EPIS(P16, 1, P32, P32, 8)
  return launch_dslash_p16h(recon, VP, OP, NS, EPI, lanes, nblocks, st, a, kptr);
}
}  // namespace stag
