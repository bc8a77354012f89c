// PBF link-storage instantiations of the half operator with PBF Krylov
// vectors and a per-site scale (STAG_HALF_VECTORS, STAG_ROUND_OUTPUT).
#include "dslash_inst.cuh"
namespace stag {
cudaError_t launch_dslash_pbfh(int recon, int VP, int OP, int NS, int EPI, int lanes, int nblocks,
                               cudaStream_t st, const DsArgs &a, const void **kptr) {
  STAG_DS_EPIS(PBF, 0, PBF, PBF, 1)
  STAG_DS_EPIS(PBF, 0, PBF, PBF, 4)
  STAG_DS_EPIS(PBF, 0, PBF, PBF, 8)
  STAG_DS_EPIS(PBF, 1, PBF, PBF, 1)
  STAG_DS_EPIS(PBF, 1, PBF, PBF, 4)
  STAG_DS_EPIS(PBF, 1, PBF, PBF, 8)
  return cudaErrorNotSupported;
}
}  // namespace stag
