// P16 link-storage instantiations of the half operator: vectors stored at
// P16 with a per-site scale (the solver), or FP32 vectors (the operator calls
// of the C ABI, whose output is returned unrounded).
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_p16(int recon, int VP, int OP, int NS, int EPI, int nblocks,
                              cudaStream_t st, const DsArgs &a) {
  STAG_DS_EPIS(P16, 0, P16, P16, 1)
  STAG_DS_EPIS(P16, 0, P16, P16, 4)
  STAG_DS_EPIS(P16, 0, P16, P16, 8)
  STAG_DS_EPIS(P16, 1, P16, P16, 1)
  STAG_DS_EPIS(P16, 1, P16, P16, 4)
  STAG_DS_EPIS(P16, 1, P16, P16, 8)
  STAG_DS_CASE(P16, 0, P32, P32, 1, EPI_PLAIN)
  STAG_DS_CASE(P16, 0, P32, P32, 1, EPI_MDAGM)
  STAG_DS_CASE(P16, 1, P32, P32, 1, EPI_PLAIN)
  STAG_DS_CASE(P16, 1, P32, P32, 1, EPI_MDAGM)
  return cudaErrorNotSupported;
}
}  // namespace stag
