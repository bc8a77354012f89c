// FP64 instantiations of the half operator: the FP64 CG and the reliable update.
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p64(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                              cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(P64, 0, P64, P64, 1)
  STAG_DS_EPIS(P64, 0, P64, P64, 4)
  STAG_DS_CASE(P64, 0, P64, P64, 1, EPI_RESID)
  STAG_DS_CASE(P64, 0, P64, P64, 4, EPI_RESID)
  STAG_DS_CASE(P64, 0, P64, P32, 1, EPI_RESID)
  STAG_DS_CASE(P64, 0, P64, P32, 4, EPI_RESID)
  return cudaErrorNotSupported;
}
}  // namespace stag
