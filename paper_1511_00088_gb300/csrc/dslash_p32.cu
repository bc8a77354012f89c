// FP32 instantiations of the half operator (full and reconstruct-12 links).
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p32(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(P32, 0, P32, P32, 1)
  STAG_DS_EPIS(P32, 0, P32, P32, 4)
  STAG_DS_EPIS(P32, 0, P32, P32, 8)
  STAG_DS_EPIS(P32, 1, P32, P32, 1)
  STAG_DS_EPIS(P32, 1, P32, P32, 4)
  STAG_DS_EPIS(P32, 1, P32, P32, 8)
  return cudaErrorNotSupported;
}
}  // namespace stag
