// PBF link-storage instantiations of the half operator: vectors stored at
// PBF with a per-site scale (the solver), or FP32 vectors (the operator calls
// of the C ABI, whose output is returned unrounded).
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_pbf(int recon, int VP, int OP, int NS, int EPI, int nblocks,
                              cudaStream_t st, const DsArgs &a) {
  STAG_DS_EPIS(PBF, 0, PBF, PBF, 1)
  STAG_DS_EPIS(PBF, 0, PBF, PBF, 4)
  STAG_DS_EPIS(PBF, 0, PBF, PBF, 8)
  STAG_DS_EPIS(PBF, 1, PBF, PBF, 1)
  STAG_DS_EPIS(PBF, 1, PBF, PBF, 4)
  STAG_DS_EPIS(PBF, 1, PBF, PBF, 8)
  STAG_DS_CASE(PBF, 0, P32, P32, 1, EPI_PLAIN)
  STAG_DS_CASE(PBF, 0, P32, P32, 1, EPI_MDAGM)
  STAG_DS_CASE(PBF, 1, P32, P32, 1, EPI_PLAIN)
  STAG_DS_CASE(PBF, 1, P32, P32, 1, EPI_MDAGM)
  return cudaErrorNotSupported;
}
}  // namespace stag
